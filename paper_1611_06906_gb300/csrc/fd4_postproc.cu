// Scale-image post-processing (Sec. 3.3, the paragraphs after Eq. 9): every
// vessel pixel (V = max_sigma V_sigma > theta) takes the scale of the set
// nearest to the mean scale of its vessel cross-section, which is traced along
// the eigenvector of the Hessian at the pixel's selected scale that belongs to
// the eigenvalue of largest magnitude (on equal magnitudes the negative one,
// the tie rule of the selection).  The Hessian direction is read from the N
// field of the tensor-build strips at the selected scales (N is the Hessian
// times a positive factor, so it has the same eigenvectors).
//
// The cross-section is the digital line through the pixel with one pixel per
// unit step along its major axis, the minor coordinate rounded half up, walked
// both ways from the pixel while it stays inside the image and the vessel mask,
// at most `cap` pixels per side; an isotropic Hessian keeps the pixel's scale;
// nearest-scale ties go to the smaller sigma; an index outside the scale set
// keeps its value and ends a walk like a pixel outside the mask.  Every pixel
// reads the scale image as selected and writes the result to a second index
// plane (idx2), which a copy kernel then moves into idx.
#include <cmath>
#include <cstdint>

#include "fd4_internal.h"

namespace fd4 {
namespace {

struct PostArgs {
    float sig[FD4_MAX_SIGMAS];
    int K;
    float theta;
    int cap;
};

// Unit eigenvector of [a b; b d] for its eigenvalue of largest magnitude (the
// negative one on a tie); false for equal eigenvalues.
__device__ __forceinline__ bool strong_direction(float a, float b, float d, float &ex, float &ey)
{
    const float m = 0.5f * (a + d), q = 0.5f * (a - d);
    const float r = hypotf(q, b);
    if (r == 0.0f) return false;
    float vx, vy;  // eigenvector of m + r
    if (q >= 0.0f) {
        vx = q + r;
        vy = b;
    } else {
        vx = b;
        vy = r - q;
    }
    const float n = hypotf(vx, vy);
    vx /= n;
    vy /= n;
    if (fabsf(m + r) > fabsf(m - r)) {
        ex = vx;
        ey = vy;
    } else {
        ex = -vy;
        ey = vx;
    }
    return true;
}

// 32 x 64 tiles (SHAPE_SWEEP), 256 threads: thread (column tid % 32, rows
// 8 (tid / 32) .. + 7).
__global__ void __launch_bounds__(256) k_postproc(Imgs I, PostArgs a)
{
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    __shared__ TileCache tcache;
    const int tid = threadIdx.x;
    if (tid == 0) tc_reset(tcache);
    const int ntiles = tile_count(I, SHAPE_SWEEP);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) find_tile_cached(I, SHAPE_SWEEP, t, tcache, sd, s_local);
        __syncthreads();
        const int w = sd.w, h = sd.h, pitch = sd.pitch;
        const int tiles_x = (w + 31) / 32;
        const int ty = s_local / tiles_x;
        const int x = (s_local - ty * tiles_x) * 32 + (tid & 31), yb = ty * 64 + (tid >> 5) * 8;
        if (x >= w) continue;
        for (int j = 0; j < 8; ++j) {
            const int y = yb + j;
            if (y >= h) break;
            const size_t p = (size_t)y * pitch + x;
            const int s0 = sd.idx[p];
            int out = s0;
            float ex, ey;
            const float4 n = sd.nfield[p];
            if (s0 < a.K && sd.vmax[p] > a.theta && strong_direction(n.x, n.y, n.z, ex, ey)) {
                const float mx = fmaxf(fabsf(ex), fabsf(ey));
                const float sx = ex / mx, sy = ey / mx;  // one of them is +-1
                float sum = a.sig[s0];
                int cnt = 1;
                for (int dir = -1; dir <= 1; dir += 2)
                    for (int k = 1; k <= a.cap; ++k) {
                        const float fk = (float)(dir * k);
                        const int qx = x + (int)floorf(fk * sx + 0.5f), qy = y + (int)floorf(fk * sy + 0.5f);
                        if (qx < 0 || qy < 0 || qx >= w || qy >= h) break;
                        const size_t q = (size_t)qy * pitch + qx;
                        const int sq = sd.idx[q];
                        if (!(sd.vmax[q] > a.theta) || sq >= a.K) break;
                        sum += a.sig[sq];
                        ++cnt;
                    }
                const float mean = sum / (float)cnt;
                int arg = 0;
                float best = fabsf(a.sig[0] - mean);
                for (int s = 1; s < a.K; ++s) {
                    const float dd = fabsf(a.sig[s] - mean);
                    if (dd < best) {
                        best = dd;
                        arg = s;
                    }
                }
                out = arg;
            }
            sd.idx2[p] = (uint8_t)out;
        }
    }
}

__global__ void __launch_bounds__(256) k_copy_idx2(Imgs I)
{
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    __shared__ TileCache tcache;
    const int tid = threadIdx.x;
    if (tid == 0) tc_reset(tcache);
    const int ntiles = tile_count(I, SHAPE_SWEEP);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) find_tile_cached(I, SHAPE_SWEEP, t, tcache, sd, s_local);
        __syncthreads();
        const int tiles_x = (sd.w + 31) / 32;
        const int ty = s_local / tiles_x;
        const int x = (s_local - ty * tiles_x) * 32 + (tid & 31), yb = ty * 64 + (tid >> 5) * 8;
        if (x >= sd.w) continue;
        for (int j = 0; j < 8 && yb + j < sd.h; ++j) {
            const size_t p = (size_t)(yb + j) * sd.pitch + x;
            sd.idx[p] = sd.idx2[p];
        }
    }
}

}  // namespace

// The post-processing of every image of B from its idx (selected scales),
// vmax and u: N at the selected scales (tensor-build strips into nfield), the
// cross-section walk into idx2, and the copy back into idx.
int launch_postprocess_batch(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                             cudaStream_t st)
{
    if (n_sigma < 1 || n_sigma > FD4_MAX_SIGMAS) return 1;
    if (launch_tensor_strips(B, h_sigmas, n_sigma, p, st)) return 1;
    PostArgs a;
    float smax = h_sigmas[0];
    for (int s = 0; s < FD4_MAX_SIGMAS; ++s) a.sig[s] = s < n_sigma ? h_sigmas[s] : 0.0f;
    for (int s = 1; s < n_sigma; ++s) smax = h_sigmas[s] > smax ? h_sigmas[s] : smax;
    a.K = n_sigma;
    a.theta = p.theta;
    a.cap = (int)std::ceil(4.0 * (double)smax);
    Imgs I = B.I;
    I.tiles = B.tiles[SHAPE_SWEEP];
    const int grid = persistent_grid((const void *)k_postproc, 256, 0, I.tiles);
    k_postproc<<<grid, 256, 0, st>>>(I, a);
    const int grid2 = persistent_grid((const void *)k_copy_idx2, 256, 0, I.tiles);
    k_copy_idx2<<<grid2, 256, 0, st>>>(I);
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace fd4
