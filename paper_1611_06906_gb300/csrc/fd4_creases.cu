// Crease extraction (Sec. 4, ridge and valley extraction): the zero contour of
// d = det(g | Hg), g the gradient and H the Hessian of u_sigma, by marching
// squares.  A tile kernel computes d and the strongest Hessian eigenvalue nu
// at every pixel (Gaussian derivatives at one scale, the taps and mirror
// border of the selection); one thread per cell then emits the cell's
// segments, kept where the mean nu of the cell's corners has the crease's
// sign (ridges negative, valleys positive; both: non-zero).  A saddle cell is
// resolved by the mean of its corners.  Segments are appended in any order
// (one counter atomic per warp), each with the key 2 * cell + k that orders
// them as the cell walk would.
#include <cmath>
#include <cstdint>

#include "fd4_internal.h"

namespace fd4 {
namespace {

constexpr int CT = 32;  // output tile side

template <int R>
struct CreaseTaps {
    float w0[2 * R + 1], w1[2 * R + 1], w2[2 * R + 1];  // tap i at offset i - R
};

__device__ __forceinline__ int cr_mirror(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

// One 32 x 32 output tile per block, 256 threads.
template <int R>
__global__ void __launch_bounds__(256) k_crease_field(const float *u, int w, int h, int pitch, CreaseTaps<R> tp,
                                                       float2 *field)
{
    constexpr int NI = CT + 2 * R;
    __shared__ float sin_[NI][NI + 1];
    __shared__ float r0[NI][CT + 1], r1[NI][CT + 1], r2[NI][CT + 1];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * CT, y0 = blockIdx.y * CT;
    for (int i = tid; i < NI * NI; i += 256) {
        const int ry = i / NI, rx = i - ry * NI;
        sin_[ry][rx] = u[(size_t)cr_mirror(y0 - R + ry, h) * pitch + cr_mirror(x0 - R + rx, w)];
    }
    __syncthreads();
    for (int i = tid; i < NI * CT; i += 256) {  // row pass: smoothing, d/dx, d2/dx2 along x
        const int ry = i / CT, x = i - ry * CT;
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) {
            const float v = sin_[ry][x + k];
            a = fmaf(tp.w0[k], v, a);
            b = fmaf(tp.w1[k], v, b);
            c = fmaf(tp.w2[k], v, c);
        }
        r0[ry][x] = a;
        r1[ry][x] = b;
        r2[ry][x] = c;
    }
    __syncthreads();
    const int x = tid & 31;
    for (int j = tid >> 5; j < CT; j += 8) {  // column pass
        const int gx = x0 + x, gy = y0 + j;
        if (gx >= w || gy >= h) continue;
        float ux = 0.f, uy = 0.f, uxx = 0.f, uxy = 0.f, uyy = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) {
            ux = fmaf(tp.w0[k], r1[j + k][x], ux);
            uy = fmaf(tp.w1[k], r0[j + k][x], uy);
            uxx = fmaf(tp.w0[k], r2[j + k][x], uxx);
            uxy = fmaf(tp.w1[k], r1[j + k][x], uxy);
            uyy = fmaf(tp.w2[k], r0[j + k][x], uyy);
        }
        const float hgx = fmaf(uxx, ux, uxy * uy), hgy = fmaf(uxy, ux, uyy * uy);
        const float d = fmaf(ux, hgy, -uy * hgx);
        const float m = 0.5f * (uxx + uyy), rr = hypotf(0.5f * (uxx - uyy), uxy);
        field[(size_t)gy * pitch + gx] = make_float2(d, m > 0.0f ? m + rr : m - rr);
    }
}

// One thread per cell (i, j): corners (i, j), (i+1, j), (i+1, j+1), (i, j+1).
// The segments of a warp are appended with one atomic on the counter (an
// inclusive scan of the lanes' counts), so no thread leaves before the scan.
__global__ void __launch_bounds__(256) k_marching(const float2 *field, int w, int h, int pitch, int mode,
                                                  float4 *segs, int *keys, int max_segs, int *count)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 32 + lane, j = blockIdx.y * 8 + (threadIdx.x >> 5);
    int ns = 0, e0[2] = {0, 0}, e1[2] = {0, 0};
    float ex[4], ey[4];  // crossings on the edges top (0-1), right (1-2), bottom (3-2), left (0-3)
    if (i + 1 < w && j + 1 < h) {
        const float2 f0 = field[(size_t)j * pitch + i], f1 = field[(size_t)j * pitch + i + 1];
        const float2 f2 = field[(size_t)(j + 1) * pitch + i + 1], f3 = field[(size_t)(j + 1) * pitch + i];
        const float c[4] = {f0.x, f1.x, f2.x, f3.x};
        const int cs = (c[0] > 0.0f) | (c[1] > 0.0f) << 1 | (c[2] > 0.0f) << 2 | (c[3] > 0.0f) << 3;
        const float nm = 0.25f * (f0.y + f1.y + f2.y + f3.y);
        const bool keep = (mode == FD4_RIDGE && nm < 0.0f) || (mode == FD4_VALLEY && nm > 0.0f) ||
                          (mode == FD4_BOTH && nm != 0.0f);
        if (cs != 0 && cs != 15 && keep) {
            ex[0] = i + c[0] / (c[0] - c[1]);
            ey[0] = (float)j;
            ex[1] = (float)(i + 1);
            ey[1] = j + c[1] / (c[1] - c[2]);
            ex[2] = i + c[3] / (c[3] - c[2]);
            ey[2] = (float)(j + 1);
            ex[3] = (float)i;
            ey[3] = j + c[0] / (c[0] - c[3]);
            if (cs == 5 || cs == 10) {  // saddle
                const float mean = 0.25f * (c[0] + c[1] + c[2] + c[3]);
                const bool cut02 = (cs == 5) != (mean > 0.0f);
                if (cut02) {
                    e0[0] = 0; e1[0] = 3; e0[1] = 1; e1[1] = 2;
                } else {
                    e0[0] = 0; e1[0] = 1; e0[1] = 2; e1[1] = 3;
                }
                ns = 2;
            } else {
                const int P0[4] = {0, 1, 3, 0}, P1[4] = {1, 2, 2, 3};
                int nc = 0;
                for (int e = 0; e < 4; ++e)
                    if ((c[P0[e]] > 0.0f) != (c[P1[e]] > 0.0f)) {
                        if (nc == 0) e0[0] = e;
                        else e1[0] = e;
                        ++nc;
                    }
                ns = 1;
            }
        }
    }
    int incl = ns;  // inclusive scan of the warp's counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int base = 0;
    if (lane == 31 && incl > 0) base = atomicAdd(count, incl);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - ns;
    for (int k = 0; k < ns; ++k)
        if (base + k < max_segs) {
            segs[base + k] = make_float4(ex[e0[k]], ey[e0[k]], ex[e1[k]], ey[e1[k]]);
            keys[base + k] = 2 * (j * (w - 1) + i) + k;
        }
}

template <int R>
int launch_field(const float *d_u, int w, int h, int pitch, const GaussTaps &g, float2 *field, cudaStream_t st)
{
    CreaseTaps<R> tp;
    const float *src[3] = {g.w0, g.w1, g.w2};
    float *dst[3] = {tp.w0, tp.w1, tp.w2};
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i <= 2 * R; ++i) {
            const int o = i - R;
            dst[k][i] = (o >= -g.r && o <= g.r) ? src[k][o + g.r] : 0.0f;
        }
    const dim3 grid((w + CT - 1) / CT, (h + CT - 1) / CT);
    k_crease_field<R><<<grid, 256, 0, st>>>(d_u, w, h, pitch, tp, field);
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace

// d and nu into the workspace field, then the segments; *d_count is cleared
// first and ends as the number of segments found (only max_segs are written).
int launch_creases(const float *d_u, int w, int h, int pitch, float sigma, int mode, float *d_segs, int *d_keys,
                   int max_segs, int *d_count, void *d_ws, cudaStream_t st)
{
    GaussTaps g;
    if (gauss_taps(sigma, &g) != FD4_OK || g.r > 16) return 1;
    float2 *field = (float2 *)d_ws;
    const int R = (g.r + 3) / 4 * 4;
    int rc = 1;
    switch (R) {
    case 4: rc = launch_field<4>(d_u, w, h, pitch, g, field, st); break;
    case 8: rc = launch_field<8>(d_u, w, h, pitch, g, field, st); break;
    case 12: rc = launch_field<12>(d_u, w, h, pitch, g, field, st); break;
    case 16: rc = launch_field<16>(d_u, w, h, pitch, g, field, st); break;
    default: rc = 1;
    }
    if (rc) return 1;
    if (cudaMemsetAsync(d_count, 0, sizeof(int), st) != cudaSuccess) return 1;
    const dim3 grid((w + 31) / 32, (h + 7) / 8);
    k_marching<<<grid, 256, 0, st>>>(field, w, h, pitch, mode, (float4 *)d_segs, d_keys, max_segs, d_count);
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace fd4
