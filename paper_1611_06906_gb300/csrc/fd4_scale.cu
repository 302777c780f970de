// Gaussian scale space, vesselness scale selection and the diffusion-tensor
// build (Sec. 3.1 Eq. 6, Sec. 3.2 Eq. 7-8, Sec. 3.3 Eq. 9).
//
// One tile kernel computes the derivatives of u_sigma = u * G_sigma for a
// 32 x 64 output tile: the tile plus a mirror-extended halo of r = ceil(4 sigma)
// pixels is staged in shared memory, a row pass applies the smoothing, first-
// and second-derivative taps along x, and a column pass combines them into
// u_x, u_y, u_xx, u_xy, u_yy.  Both passes keep a sliding register window so
// that each shared-memory load feeds eight outputs.  The work is FP32 FMA
// bound (about 2 (2r+1) (3 + 5) FMAs per pixel and scale).
#include <cstdint>

#include "fd4_internal.h"

namespace fd4 {
namespace {

constexpr int TX = 32;        // output tile width
constexpr int TY = 64;        // output tile height
constexpr int VR = 8;         // row pass: outputs per thread along x
constexpr int VC = 8;         // column pass: outputs per thread along y
constexpr int NT = 256;       // threads per block
constexpr int RS = TX + 1;    // row-pass output stride (conflict-free column reads)

static_assert(TX / VR * 8 == 32, "row pass maps 8 rows x 4 segments to a warp");
static_assert(TX * (TY / VC) == NT, "column pass: one unit per thread");

__host__ __device__ inline int in_stride(int r)
{
    // >= TX + 2r and == 1 mod 32: the 8 rows a warp touches in the row pass
    // start in 8 different banks.
    return ((TX + 2 * r - 1 + 31) / 32) * 32 + 1;
}

__host__ __device__ inline size_t tile_smem_bytes(int r)
{
    const int rows = TY + 2 * r;
    return sizeof(float) * ((size_t)3 * (2 * r + 1) + (size_t)rows * in_stride(r) + (size_t)3 * rows * RS);
}

__device__ __forceinline__ int mirror(int i, int n)
{
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

// a d - b^2 with Kahan's fma compensation (error analysed by Jeannerod,
// Louvet and Muller, Math. Comp. 2013): accurate even under cancellation.
__device__ __forceinline__ float det2_sym(float a, float b, float d)
{
    const float bb = b * b;
    const float err = fmaf(-b, b, bb);
    return fmaf(a, d, -bb) + err;
}

struct SelectOut {
    float *vp;          // K planes: exp(-R_B^2/(2 beta^2)), 0 for the wrong polarity
    float *s2;          // K planes: S^2
    size_t plane;       // elements per plane
    int s;              // scale index
    float scale4;       // sigma^(4 gamma)
    float inv2b2;       // 1 / (2 beta^2)
    int mode;
    unsigned *max_s2;   // float bits
};

struct TensorOut {
    const uint8_t *idx;
    float4 *nfield;     // (Nxx, Nxy, Nyy, 0)
    int s;
    int grad_sq;
};

enum { OUT_SELECT = 0, OUT_TENSOR = 1 };

template <int OUT>
__global__ void __launch_bounds__(NT) k_gauss_tile(const float *__restrict__ img, int w, int h, int pitch,
                                                   GaussTaps taps, SelectOut so, TensorOut to)
{
    extern __shared__ float smem[];
    const int r = taps.r;
    const int nt = 2 * r + 1;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (OUT == OUT_TENSOR) {
        // only tiles holding a pixel whose selected scale is this one do work
        int any = 0;
        for (int i = tid; i < TX * TY; i += NT) {
            const int x = x0 + (i & (TX - 1)), y = y0 + i / TX;
            if (x < w && y < h && to.idx[(size_t)y * pitch + x] == to.s) any = 1;
        }
        if (!__syncthreads_or(any)) return;
    }

    const int S = in_stride(r);
    const int rows = TY + 2 * r;
    float *wt = smem;                    // w0 | w1 | w2, nt each
    float *tin = wt + 3 * nt;            // rows x S input with halo
    float *trow = tin + rows * S;        // 3 fields x rows x RS
    for (int i = tid; i < nt; i += NT) {
        wt[i] = taps.w0[i];
        wt[nt + i] = taps.w1[i];
        wt[2 * nt + i] = taps.w2[i];
    }
    const int in_w = TX + 2 * r;
    for (int ry = warp; ry < rows; ry += NT / 32) {
        const float *src = img + (size_t)mirror(y0 - r + ry, h) * pitch;
        for (int rx = lane; rx < in_w; rx += 32)
            tin[ry * S + rx] = __ldg(src + mirror(x0 - r + rx, w));
    }
    __syncthreads();

    // Row pass: three filtered fields along x for every staged row.
    for (int u = tid; u < rows * (TX / VR); u += NT) {
        const int ry = u >> 2, xo = (u & 3) * VR;
        const float *src = tin + ry * S + xo;
        float a0[VR], a1[VR], a2[VR], win[VR];
#pragma unroll
        for (int j = 0; j < VR; ++j) {
            a0[j] = a1[j] = a2[j] = 0.0f;
            win[j] = src[j];
        }
        for (int k = 0; k < nt; ++k) {
            const float c0 = wt[k], c1 = wt[nt + k], c2 = wt[2 * nt + k];
#pragma unroll
            for (int j = 0; j < VR; ++j) {
                a0[j] = fmaf(c0, win[j], a0[j]);
                a1[j] = fmaf(c1, win[j], a1[j]);
                a2[j] = fmaf(c2, win[j], a2[j]);
            }
#pragma unroll
            for (int j = 0; j < VR - 1; ++j) win[j] = win[j + 1];
            if (k + 1 < nt) win[VR - 1] = src[VR + k];
        }
        float *d0 = trow + ry * RS + xo;
#pragma unroll
        for (int j = 0; j < VR; ++j) {
            d0[j] = a0[j];
            d0[rows * RS + j] = a1[j];
            d0[2 * rows * RS + j] = a2[j];
        }
    }
    __syncthreads();

    // Column pass: thread owns column ox, rows oy0 .. oy0+VC-1 of the tile.
    const int ox = tid & 31, oy0 = (tid >> 5) * VC;
    float uxx[VC], uxy[VC], uyy[VC], ux[VC], uy[VC];
    {   // field 2 (second derivative along x) smoothed along y -> u_xx
        const float *src = trow + 2 * rows * RS + oy0 * RS + ox;
        float win[VC];
#pragma unroll
        for (int j = 0; j < VC; ++j) {
            uxx[j] = 0.0f;
            win[j] = src[j * RS];
        }
        for (int k = 0; k < nt; ++k) {
            const float c0 = wt[k];
#pragma unroll
            for (int j = 0; j < VC; ++j) uxx[j] = fmaf(c0, win[j], uxx[j]);
#pragma unroll
            for (int j = 0; j < VC - 1; ++j) win[j] = win[j + 1];
            if (k + 1 < nt) win[VC - 1] = src[(VC + k) * RS];
        }
    }
    {   // field 1 (first derivative along x): smoothed -> u_x, differentiated -> u_xy
        const float *src = trow + rows * RS + oy0 * RS + ox;
        float win[VC];
#pragma unroll
        for (int j = 0; j < VC; ++j) {
            ux[j] = uxy[j] = 0.0f;
            win[j] = src[j * RS];
        }
        for (int k = 0; k < nt; ++k) {
            const float c0 = wt[k], c1 = wt[nt + k];
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                ux[j] = fmaf(c0, win[j], ux[j]);
                uxy[j] = fmaf(c1, win[j], uxy[j]);
            }
#pragma unroll
            for (int j = 0; j < VC - 1; ++j) win[j] = win[j + 1];
            if (k + 1 < nt) win[VC - 1] = src[(VC + k) * RS];
        }
    }
    {   // field 0 (smoothed along x): first derivative -> u_y, second -> u_yy
        const float *src = trow + oy0 * RS + ox;
        float win[VC];
#pragma unroll
        for (int j = 0; j < VC; ++j) {
            uy[j] = uyy[j] = 0.0f;
            win[j] = src[j * RS];
        }
        for (int k = 0; k < nt; ++k) {
            const float c1 = wt[nt + k], c2 = wt[2 * nt + k];
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                uy[j] = fmaf(c1, win[j], uy[j]);
                uyy[j] = fmaf(c2, win[j], uyy[j]);
            }
#pragma unroll
            for (int j = 0; j < VC - 1; ++j) win[j] = win[j + 1];
            if (k + 1 < nt) win[VC - 1] = src[(VC + k) * RS];
        }
    }

    const int gx = x0 + ox;
    float bmax = 0.0f;
#pragma unroll
    for (int j = 0; j < VC; ++j) {
        const int gy = y0 + oy0 + j;
        if (gx >= w || gy >= h) continue;
        const size_t p = (size_t)gy * pitch + gx;
        const float a = uxx[j], b = uxy[j], d = uyy[j];
        if (OUT == OUT_SELECT) {
            // eigenvalues of H (the sigma^(2 gamma) factor cancels in R_B and
            // the sign test; S^2 picks it up as sigma^(4 gamma))
            const float m = 0.5f * (a + d);
            const float rr = hypotf(0.5f * (a - d), b);
            const float far = m > 0.0f ? m + rr : m - rr;  // larger magnitude; ties -> negative
            float vp = 0.0f;
            const bool wrong = (so.mode == FD4_RIDGE && far > 0.0f) || (so.mode == FD4_VALLEY && far < 0.0f);
            if (!wrong && far != 0.0f) {
                const float near = det2_sym(a, b, d) / far;        // cancellation-free
                const float rb = near / far;
                vp = expf(-rb * rb * so.inv2b2);
            }
            const float s2 = so.scale4 * fmaf(a, a, fmaf(2.0f * b, b, d * d));
            so.vp[so.s * so.plane + p] = vp;
            so.s2[so.s * so.plane + p] = s2;
            bmax = fmaxf(bmax, s2);
        } else {
            if (to.idx[p] != to.s) continue;
            const float g2 = fmaf(ux[j], ux[j], uy[j] * uy[j]);
            const float g = to.grad_sq ? g2 : sqrtf(g2);
            const float f = 1.0f / sqrtf(1.0f + g);
            to.nfield[p] = make_float4(f * a, f * b, f * d, 0.0f);
        }
    }
    if (OUT == OUT_SELECT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        __shared__ float wmax[NT / 32];
        if (lane == 0) wmax[warp] = bmax;
        __syncthreads();
        if (tid == 0) {
            float m = wmax[0];
            for (int i = 1; i < NT / 32; ++i) m = fmaxf(m, wmax[i]);
            atomicMax(so.max_s2, __float_as_uint(m));
        }
    }
}

// Second selection pass: V = vp (1 - exp(-S^2 / (2 c^2))) per scale, argmax with
// ties to the smaller scale (strict comparison in increasing sigma order).
__global__ void k_select_argmax(const float *__restrict__ vp, const float *__restrict__ s2, size_t plane,
                                int K, int w, int h, int pitch, const unsigned *max_s2, float c_user,
                                uint8_t *idx, float *vmax)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= w || y >= h) return;
    float k2;  // 1 / (2 c^2)
    if (c_user > 0.0f) {
        k2 = 0.5f / (c_user * c_user);
    } else {
        const float m = __uint_as_float(*max_s2);  // max S^2 = (2c)^2
        k2 = m > 0.0f ? 2.0f / m : 0.0f;
    }
    const size_t p = (size_t)y * pitch + x;
    float best = -1.0f;
    int arg = 0;
    for (int s = 0; s < K; ++s) {
        float v = __ldg(vp + s * plane + p);
        v = (v > 0.0f && k2 > 0.0f) ? v * -expm1f(-__ldg(s2 + s * plane + p) * k2) : 0.0f;
        if (v > best) {
            best = v;
            arg = s;
        }
    }
    idx[p] = (uint8_t)arg;
    if (vmax) vmax[p] = best;
}

__device__ __forceinline__ float pm_mu(float nu, float lambda, int mode)
{
    if ((mode == FD4_RIDGE && nu >= 0.0f) || (mode == FD4_VALLEY && nu <= 0.0f)) return 1.0f;
    const float q = nu / lambda;
    return 1.0f / fmaf(q, q, 1.0f);
}

constexpr int FX = 32, FY = 8;   // tensor-finish tile

// N_rho = G_rho * N (mirror border), closed-form eigen-decomposition and
// Perona-Malik diffusivities -> (cos 2t, sin 2t, mu1, mu2), e1 for nu1 >= nu2.
__global__ void __launch_bounds__(FX * FY) k_tensor_finish(const float4 *__restrict__ nf, int w, int h, int pitch,
                                                            RhoTaps taps, float lambda, int mode, float4 *out)
{
    __shared__ float4 sin_[FY + 2 * kMaxRhoRadius][FX + 2 * kMaxRhoRadius];
    __shared__ float4 srow[FY + 2 * kMaxRhoRadius][FX];
    const int r = taps.r;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * FY;
    const int tid = threadIdx.x;
    const int rows = FY + 2 * r, cols = FX + 2 * r;
    for (int i = tid; i < rows * cols; i += FX * FY) {
        const int ry = i / cols, rx = i - ry * cols;
        sin_[ry][rx] = nf[(size_t)mirror(y0 - r + ry, h) * pitch + mirror(x0 - r + rx, w)];
    }
    __syncthreads();
    for (int i = tid; i < rows * FX; i += FX * FY) {
        const int ry = i / FX, rx = i - ry * FX;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k <= 2 * r; ++k) {
            const float c = taps.w0[k];
            const float4 v = sin_[ry][rx + k];
            a.x = fmaf(c, v.x, a.x);
            a.y = fmaf(c, v.y, a.y);
            a.z = fmaf(c, v.z, a.z);
        }
        srow[ry][rx] = a;
    }
    __syncthreads();
    const int tx = tid & (FX - 1), ty = tid / FX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= w || gy >= h) return;
    float a = 0.f, b = 0.f, d = 0.f;
    for (int k = 0; k <= 2 * r; ++k) {
        const float c = taps.w0[k];
        const float4 v = srow[ty + k][tx];
        a = fmaf(c, v.x, a);
        b = fmaf(c, v.y, b);
        d = fmaf(c, v.z, d);
    }
    const float m = 0.5f * (a + d), q = 0.5f * (a - d);
    const float rr = hypotf(q, b);
    const float det = det2_sym(a, b, d);
    float nu1, nu2;
    if (m > 0.0f) {
        nu1 = m + rr;
        nu2 = det / nu1;
    } else if (m < 0.0f) {
        nu2 = m - rr;
        nu1 = det / nu2;
    } else {
        nu1 = rr;
        nu2 = -rr;
    }
    float c2 = 1.0f, s2 = 0.0f;
    if (rr > 0.0f) {
        c2 = q / rr;
        s2 = b / rr;
    }
    out[(size_t)gy * pitch + gx] = make_float4(c2, s2, pm_mu(nu1, lambda, mode), pm_mu(nu2, lambda, mode));
}

int set_tile_smem()
{
    static int done = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (done == dev) return 0;
    const int bytes = (int)tile_smem_bytes(kMaxRadius);
    if (cudaFuncSetAttribute(k_gauss_tile<OUT_SELECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return 1;
    if (cudaFuncSetAttribute(k_gauss_tile<OUT_TENSOR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return 1;
    done = dev;
    return 0;
}

}  // namespace

int launch_select(const float *d_img, int w, int h, int pitch, const float *h_sigmas, int n_sigma,
                  const fd4_params &p, uint8_t *d_idx, float *d_vmax, char *ws, cudaStream_t st)
{
    if (set_tile_smem()) return 1;
    WsHeader *hdr = (WsHeader *)ws;
    const size_t plane = (size_t)h * pitch;
    const size_t pb = plane_bytes(h, pitch, 4);
    float *vp = (float *)(ws + kHeaderBytes);
    float *s2 = (float *)(ws + kHeaderBytes + (size_t)n_sigma * pb);
    const size_t pstride = pb / 4;  // plane stride in floats (>= plane)
    if (cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st) != cudaSuccess) return 1;
    const dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY);
    TensorOut to{};
    for (int s = 0; s < n_sigma; ++s) {
        GaussTaps taps;
        if (gauss_taps(h_sigmas[s], &taps) != FD4_OK) return 1;
        SelectOut so;
        so.vp = vp;
        so.s2 = s2;
        so.plane = pstride;
        so.s = s;
        so.scale4 = (float)pow((double)h_sigmas[s], 4.0 * p.gamma);
        so.inv2b2 = (float)(1.0 / (2.0 * (double)p.beta * p.beta));
        so.mode = p.mode;
        so.max_s2 = &hdr->max_s2;
        k_gauss_tile<OUT_SELECT><<<grid, NT, tile_smem_bytes(taps.r), st>>>(d_img, w, h, pitch, taps, so, to);
    }
    (void)plane;
    k_select_argmax<<<dim3((w + 127) / 128, h), 128, 0, st>>>(vp, s2, pstride, n_sigma, w, h, pitch,
                                                             &hdr->max_s2, p.c, d_idx, d_vmax);
    return cudaGetLastError() != cudaSuccess;
}

int launch_tensor(const float *d_u, int w, int h, int pitch, const uint8_t *d_idx, const float *h_sigmas,
                  int n_sigma, const fd4_params &p, float *d_tensor, char *ws, cudaStream_t st)
{
    if (set_tile_smem()) return 1;
    float4 *nf = (float4 *)(ws + kHeaderBytes);
    // pixels whose index is out of range keep N = 0 (isotropic, mu = 1)
    if (cudaMemsetAsync(nf, 0, (size_t)h * pitch * sizeof(float4), st) != cudaSuccess) return 1;
    const dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY);
    SelectOut so{};
    for (int s = 0; s < n_sigma; ++s) {
        GaussTaps taps;
        if (gauss_taps(h_sigmas[s], &taps) != FD4_OK) return 1;
        TensorOut to;
        to.idx = d_idx;
        to.nfield = nf;
        to.s = s;
        to.grad_sq = p.grad_norm_squared;
        k_gauss_tile<OUT_TENSOR><<<grid, NT, tile_smem_bytes(taps.r), st>>>(d_u, w, h, pitch, taps, so, to);
    }
    RhoTaps rt;
    if (rho_taps(p.rho, &rt) != FD4_OK) return 1;
    k_tensor_finish<<<dim3((w + FX - 1) / FX, (h + FY - 1) / FY), FX * FY, 0, st>>>(
        nf, w, h, pitch, rt, p.lambda, p.mode, (float4 *)d_tensor);
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace fd4
