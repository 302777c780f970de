// Gaussian scale space, vesselness scale selection and the diffusion-tensor
// build (Sec. 3.1 Eq. 6, Sec. 3.2 Eq. 7-8, Sec. 3.3 Eq. 9).
//
// k_scale_sweep computes the derivatives of u_sigma = u * G_sigma for every
// scale of the set on a 32 x 64 output tile in one block: the tile plus a
// mirror-extended halo of the largest radius is staged in shared memory once,
// then for each scale a row pass applies the smoothing, first- and
// second-derivative taps along x and a column pass combines them into
// u_x, u_y, u_xx, u_xy, u_yy.  Both passes keep register windows that are
// refilled four taps at a time (one 16-byte shared load in the row pass), so
// the inner loops are almost pure FMA.  The work is FP32-FMA bound: about
// 3 (2R+4)(1 + (2R+8)/64) + 5 (2R+4) FMAs per pixel and scale, R = ceil(4 sigma)
// rounded up to a multiple of 4.  It serves the selection restricted to a
// list of tiles (the learned selector's fallback); whole images are selected by
// the per-scale strip kernels of fd4_tensor.cu, which compute the same sums in
// the same order.
#include <cstdint>

#include "fd4_internal.h"

namespace fd4 {
namespace {

constexpr int TX = 32;        // output tile width
constexpr int TY = 64;        // output tile height
constexpr int VR = 8;         // row pass: outputs per thread along x
constexpr int VC = 4;         // column pass: outputs per thread along y
constexpr int NT = 512;       // threads per block
constexpr int RS = TX + 1;    // row-pass output stride (conflict-free column reads)
constexpr int kMaxSweep = 16; // scales per launch
constexpr int kSweepFloats = kMaxSweep * 3 * (2 * kMaxRadius + 4);

static_assert(TX * (TY / VC) == NT, "column pass: one unit per thread");

// Taps of up to kMaxSweep scales.  Scale s uses the padded radius R[s] (a
// multiple of 4, >= ceil(4 sigma)); its three kernels w0, w1, w2 (smoothing,
// first and second derivative, correlation weights) each hold L = 2R+4
// entries at w[off[s] + k*L + i], entry i being the tap at offset i - R (zero
// beyond the true radius).
struct SweepTaps {
    int K;                    // scales in this launch
    int K_total;              // size of the whole scale set
    int s0;                   // index of this launch's first scale in the set
    int Rmax;                 // max R[s]
    int R[kMaxSweep];
    int off[kMaxSweep];
    float scale4[kMaxSweep];  // sigma^(4 gamma)
    int wfloats;              // used entries of w (multiple of 4)
    float w[kSweepFloats];
};

__host__ __device__ inline int sweep_in_stride(int Rmax)
{
    // >= TX + 2 Rmax + 4 (the row pass reads up to column 35 + 2 Rmax) and
    // == 4 mod 8: 16-byte aligned rows, and the 16-byte loads of two adjacent
    // rows (one quarter-warp phase) fall in different bank quads.
    const int need = TX + 2 * Rmax + 4;
    return ((need - 4 + 7) / 8) * 8 + 4;
}

// the column pass reads staged rows up to 67 + 2 Rmax
__host__ __device__ inline int sweep_rows(int Rmax) { return TY + 2 * Rmax + 4; }

__host__ __device__ inline size_t sweep_smem_bytes(int Rmax, int wfloats)
{
    const int rows = sweep_rows(Rmax);
    return sizeof(float) * ((size_t)wfloats + (size_t)rows * sweep_in_stride(Rmax) + (size_t)3 * rows * RS);
}

__device__ __forceinline__ int mirror(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;  // the common case: no reflection
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

// Column pass of one field over the 12-row register window: acc_a += wa * field
// (and acc_b += wb * field when TWO), VC outputs down one column.
template <bool TWO>
__device__ __forceinline__ void column_pass(const float *src, const float *wa, const float *wb, int nch,
                                            float (&acc_a)[VC], float (&acc_b)[VC])
{
    float win[VC + 4];
#pragma unroll
    for (int q = 0; q < VC + 4; ++q) win[q] = src[q * RS];
#pragma unroll
    for (int j = 0; j < VC; ++j) {
        acc_a[j] = 0.0f;
        if (TWO) acc_b[j] = 0.0f;
    }
    for (int ch = 0; ch < nch; ++ch) {
        const float4 A = *reinterpret_cast<const float4 *>(wa + 4 * ch);
        float4 B = make_float4(0.f, 0.f, 0.f, 0.f);
        if (TWO) B = *reinterpret_cast<const float4 *>(wb + 4 * ch);
        const float av[4] = {A.x, A.y, A.z, A.w};
        const float bv[4] = {B.x, B.y, B.z, B.w};
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                acc_a[j] = fmaf(av[ii], win[j + ii], acc_a[j]);
                if (TWO) acc_b[j] = fmaf(bv[ii], win[j + ii], acc_b[j]);
            }
        }
        if (ch + 1 < nch) {
#pragma unroll
            for (int q = 0; q < VC; ++q) win[q] = win[q + 4];
#pragma unroll
            for (int q = 0; q < 4; ++q) win[VC + q] = src[(4 * ch + VC + 4 + q) * RS];
        }
    }
}

__global__ void __launch_bounds__(NT, 2) k_scale_sweep(Imgs I, SweepTaps taps, float inv2b2, int mode)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    const int Rmax = taps.Rmax;
    const int S = sweep_in_stride(Rmax);
    const int rows = sweep_rows(Rmax);
    const int in_w = TX + 2 * Rmax + 4;
    float *wt = smem;                        // taps
    float *tin = wt + taps.wfloats;          // rows x S staged input
    float *trow = tin + rows * S;            // 3 fields x rows x RS
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < taps.wfloats; i += NT) wt[i] = taps.w[i];

    const int ntiles = tile_count(I, SHAPE_SWEEP);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();   // the previous tile is done with shared memory
    if (tid == 0) find_tile(I, SHAPE_SWEEP, t, sd, s_local);
    __syncthreads();
    const int w = sd.w, h = sd.h, pitch = sd.pitch;
    const int tiles_x = (w + TX - 1) / TX;
    const int x0 = (s_local % tiles_x) * TX, y0 = (s_local / tiles_x) * TY;
    const float *img = sd.in;
    for (int ry = warp; ry < rows; ry += NT / 32) {
        const float *src = img + (size_t)mirror(y0 - Rmax + ry, h) * pitch;
        for (int rx = lane; rx < in_w; rx += 32) tin[ry * S + rx] = __ldg(src + mirror(x0 - Rmax + rx, w));
    }

    const int ox = tid & 31, oy0 = (tid >> 5) * VC;
    const int gx = x0 + ox;
    __syncthreads();

    float bmax = 0.0f;
    for (int s = 0; s < taps.K; ++s) {
        const int R = taps.R[s];
        const int L = 2 * R + 4, nch = L / 4;
        const int off = Rmax - R;
        const float *w0 = wt + taps.off[s], *w1 = w0 + L, *w2 = w1 + L;

        // Row pass: three fields along x on staged rows [off, off + TY + 2R + 4),
        // four 8-column chunks per row.
        const int nrows = TY + 2 * R + 4;
        for (int u = tid; u < nrows * (TX / VR); u += NT) {
            const int q = u / (TX / VR), sy = off + q, xo = (u - q * (TX / VR)) * VR;
            const float *src = tin + sy * S + xo + off;
            float win[VR + 4];
            {
                const float4 a = *reinterpret_cast<const float4 *>(src);
                const float4 b = *reinterpret_cast<const float4 *>(src + 4);
                const float4 c = *reinterpret_cast<const float4 *>(src + 8);
                win[0] = a.x; win[1] = a.y; win[2] = a.z; win[3] = a.w;
                win[4] = b.x; win[5] = b.y; win[6] = b.z; win[7] = b.w;
                win[8] = c.x; win[9] = c.y; win[10] = c.z; win[11] = c.w;
            }
            float a0[VR], a1[VR], a2[VR];
#pragma unroll
            for (int j = 0; j < VR; ++j) a0[j] = a1[j] = a2[j] = 0.0f;
            for (int ch = 0; ch < nch; ++ch) {
                const float4 W0 = *reinterpret_cast<const float4 *>(w0 + 4 * ch);
                const float4 W1 = *reinterpret_cast<const float4 *>(w1 + 4 * ch);
                const float4 W2 = *reinterpret_cast<const float4 *>(w2 + 4 * ch);
                const float c0[4] = {W0.x, W0.y, W0.z, W0.w};
                const float c1[4] = {W1.x, W1.y, W1.z, W1.w};
                const float c2[4] = {W2.x, W2.y, W2.z, W2.w};
#pragma unroll
                for (int ii = 0; ii < 4; ++ii) {
#pragma unroll
                    for (int j = 0; j < VR; ++j) {
                        a0[j] = fmaf(c0[ii], win[j + ii], a0[j]);
                        a1[j] = fmaf(c1[ii], win[j + ii], a1[j]);
                        a2[j] = fmaf(c2[ii], win[j + ii], a2[j]);
                    }
                }
                if (ch + 1 < nch) {
#pragma unroll
                    for (int q = 0; q < VR; ++q) win[q] = win[q + 4];
                    const float4 d = *reinterpret_cast<const float4 *>(src + 4 * ch + 12);
                    win[8] = d.x; win[9] = d.y; win[10] = d.z; win[11] = d.w;
                }
            }
            float *d0 = trow + sy * RS + xo;
#pragma unroll
            for (int j = 0; j < VR; ++j) {
                d0[j] = a0[j];
                d0[rows * RS + j] = a1[j];
                d0[2 * rows * RS + j] = a2[j];
            }
        }
        __syncthreads();

        // Column pass: tile column ox, tile rows oy0 .. oy0 + VC - 1.
        const float *col = trow + (oy0 + off) * RS + ox;
        float uxx[VC], uxy[VC], uyy[VC];
        column_pass<false>(col + 2 * rows * RS, w0, w0, nch, uxx, uxx);      // d2/dx2, smoothed in y
        column_pass<false>(col + rows * RS, w1, w1, nch, uxy, uxy);          // d/dx, then d/dy
        column_pass<false>(col, w2, w2, nch, uyy, uyy);                      // d2/dy2 of the x-smoothed field
        __syncthreads();   // trow is rewritten by the next scale's row pass

#pragma unroll
        for (int j = 0; j < VC; ++j) {
            const int gy = y0 + oy0 + j;
            if (gx >= w || gy >= h) continue;
            const float a = uxx[j], b = uxy[j], d = uyy[j];
            {
                // eigenvalues of H (sigma^(2 gamma) cancels in R_B and the sign
                // test; S^2 picks it up as sigma^(4 gamma))
                const float m = 0.5f * (a + d);
                const float rr = hypotf(0.5f * (a - d), b);
                const float far = m > 0.0f ? m + rr : m - rr;  // larger magnitude; ties -> negative
                float vp = 0.0f;
                const bool wrong = (mode == FD4_RIDGE && far > 0.0f) || (mode == FD4_VALLEY && far < 0.0f);
                if (!wrong && far != 0.0f) {
                    const float near = det2_sym(a, b, d) / far;  // cancellation-free
                    const float rb = near / far;
                    vp = expf(-rb * rb * inv2b2);
                }
                const float s2 = taps.scale4[s] * fmaf(a, a, fmaf(2.0f * b, b, d * d));
                const size_t p = (size_t)gy * pitch + gx;
                sd.vp[(size_t)(taps.s0 + s) * sd.plane + p] = vp;
                sd.s2[(size_t)(taps.s0 + s) * sd.plane + p] = s2;
                bmax = fmaxf(bmax, s2);
            }
        }
    }

    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        if (lane == 0 && bmax > 0.0f) atomicMax(sd.max_s2, __float_as_uint(bmax));
    }
    }  // tile loop
}

// Second selection pass: V = vp (1 - exp(-S^2 / (2 c^2))) per scale, argmax with
// ties to the smaller scale (strict comparison in increasing sigma order).
// 32 x 64 tiles (SHAPE_SWEEP), 256 threads: thread (column quad tid % 8, rows
// tid / 8 and tid / 8 + 32) reads each plane as two float4, so 8 pixels' loads
// of a scale are in flight together.
__global__ void __launch_bounds__(256) k_select_argmax(Imgs I, int K, float c_user)
{
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    __shared__ TileCache tcache;
    if (threadIdx.x == 0) tc_reset(tcache);
    const int tid = threadIdx.x;
    const int qx = (tid & 7) * 4, ry = tid >> 3;
    const int ntiles = tile_count(I, SHAPE_SWEEP);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) find_tile_cached(I, SHAPE_SWEEP, t, tcache, sd, s_local);
        __syncthreads();
        const int tiles_x = (sd.w + 31) / 32;
        const int ty = s_local / tiles_x;
        const int x = (s_local - ty * tiles_x) * 32 + qx, y0 = ty * 64 + ry;
        if (x >= sd.w) continue;
        float k2;  // 1 / (2 c^2)
        if (c_user > 0.0f) {
            k2 = 0.5f / (c_user * c_user);
        } else {
            const float m = __uint_as_float(*sd.max_s2);  // max S^2 = (2c)^2
            k2 = m > 0.0f ? 2.0f / m : 0.0f;
        }
        // rows y0 and y0 + 32; a quad starting inside the row stays inside the pitch
        const bool row_ok[2] = {y0 < sd.h, y0 + 32 < sd.h};
        size_t p[2];
        p[0] = (size_t)y0 * sd.pitch + x;
        p[1] = p[0] + (size_t)32 * sd.pitch;
        float best[8];
        int arg[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            best[i] = -1.0f;
            arg[i] = 0;
        }
        for (int s = 0; s < K; ++s) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (!row_ok[r]) continue;
                const float4 v4 = __ldg(reinterpret_cast<const float4 *>(sd.vp + s * sd.plane + p[r]));
                const float4 s4 = __ldg(reinterpret_cast<const float4 *>(sd.s2 + s * sd.plane + p[r]));
                const float vv[4] = {v4.x, v4.y, v4.z, v4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float v = (vv[i] > 0.0f && k2 > 0.0f) ? vv[i] * -expm1f(-sv[i] * k2) : 0.0f;
                    if (v > best[4 * r + i]) {
                        best[4 * r + i] = v;
                        arg[4 * r + i] = s;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!row_ok[r]) continue;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (x + i >= sd.w) continue;
                sd.idx[p[r] + i] = (uint8_t)arg[4 * r + i];
                if (sd.vmax) sd.vmax[p[r] + i] = best[4 * r + i];
            }
        }
    }
}

// Perona-Malik diffusivity 1 / (1 + nu^2 / lambda^2) with ridge/valley gating;
// inv_lambda = 1 / lambda.
__device__ __forceinline__ float pm_mu(float nu, float inv_lambda, int mode)
{
    if ((mode == FD4_RIDGE && nu >= 0.0f) || (mode == FD4_VALLEY && nu <= 0.0f)) return 1.0f;
    const float q = nu * inv_lambda;
    return __fdividef(1.0f, fmaf(q, q, 1.0f));  // divisor >= 1: the fast reciprocal is within 2 ulp
}

// Tensor finish on 32 x 64 tiles (SHAPE_SWEEP), 256 threads: N_rho = G_rho * N
// (mirror border; row pass then column pass, taps in increasing order), the
// closed-form eigen-decomposition of N_rho and the Perona-Malik diffusivities
// -> (cos 2t, sin 2t, mu1, mu2), e1 for nu1 >= nu2.  The G_rho radius r is a
// template parameter (r = ceil(4 rho) <= 8).
// Each 32 x 64 tile is finished as two halves of FH = 32 rows (the smaller
// staging buffers let three blocks share an SM).
constexpr int FX = 32, FY = 64, FH = 32, FNT_T = 256;
// Row strides of the staged region and of the row-smoothed rows, in float4
// pixels: odd, so that the 16-byte accesses of eight threads on eight
// consecutive rows of one column fall in eight distinct bank groups.
template <int r>
constexpr int finish_cp() { return FX + 2 * r + 1; }
constexpr int FSR = FX + 1;

template <int r>
constexpr size_t finish_smem_bytes()
{
    return sizeof(float4) * ((size_t)2 * (FH + 2 * r) * finish_cp<r>() + (size_t)(FH + 2 * r) * FSR);
}

// cp.async (16 bytes = one pixel of N) of a half tile's N region with its mirrored halo.
template <int r>
__device__ __forceinline__ void finish_stage(const ImgDesc &d, int2 o, float4 *dst)
{
    constexpr int ROWS = FH + 2 * r, COLS = FX + 2 * r, CP = finish_cp<r>();
    const int w = d.w, h = d.h, pitch = d.pitch, x0 = o.x, y0 = o.y;
    if (x0 >= r && y0 >= r && x0 + FX + r <= w && y0 + FH + r <= h) {  // no mirrored index
        const float4 *base = d.nfield + (size_t)(y0 - r) * pitch + (x0 - r);
        for (int i = threadIdx.x; i < ROWS * COLS; i += FNT_T) {
            const int ry = i / COLS, rx = i - ry * COLS;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             (unsigned)__cvta_generic_to_shared(dst + ry * CP + rx)),
                         "l"(base + (size_t)ry * pitch + rx)
                         : "memory");
        }
    } else {
        for (int i = threadIdx.x; i < ROWS * COLS; i += FNT_T) {
            const int ry = i / COLS, rx = i - ry * COLS;
            const float4 *src = d.nfield + (size_t)mirror(y0 - r + ry, h) * pitch + mirror(x0 - r + rx, w);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             (unsigned)__cvta_generic_to_shared(dst + ry * CP + rx)),
                         "l"(src)
                         : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The origin of half hf of a finish tile, computed once by the thread that looks it up.
__device__ __forceinline__ int2 finish_origin(const ImgDesc &d, int local, int hf)
{
    const int tiles_x = (d.w + FX - 1) / FX;
    const int ty = local / tiles_x;
    return make_int2((local - ty * tiles_x) * FX, ty * FY + hf * FH);
}

// The next half tile's region is copied (cp.async, double buffer) while the
// current one is smoothed and decomposed.  Work unit u = half u % 2 of tile u / 2.
template <int r>
__global__ void __launch_bounds__(FNT_T) k_tensor_finish(Imgs I, RhoTaps taps, float lambda, int mode, int soa)
{
    constexpr int ROWS = FH + 2 * r, CP = finish_cp<r>();
    extern __shared__ __align__(16) float4 fsm4[];
    // two ROWS x CP buffers: N with the mirrored halo; then ROWS x FSR: smoothed along x
    float4 *srow = fsm4 + 2 * ROWS * CP;
    __shared__ ImgDesc sdb[2];
    __shared__ int s_localb[2];
    __shared__ int2 sorg[2];
    __shared__ TileCache tcache;
    const int tid = threadIdx.x;
    float wr[2 * r + 1];
#pragma unroll
    for (int k = 0; k <= 2 * r; ++k) wr[k] = taps.w0[k];
    const float inv_lambda = 1.0f / lambda;
    const int nunits = 2 * tile_count(I, SHAPE_SWEEP);
    int u = blockIdx.x, cur = 0;
    if (u >= nunits) return;
    if (tid == 0) {
        tc_reset(tcache);
        find_tile_cached(I, SHAPE_SWEEP, u >> 1, tcache, sdb[0], s_localb[0]);
        sorg[0] = finish_origin(sdb[0], s_localb[0], u & 1);
    }
    __syncthreads();
    finish_stage<r>(sdb[0], sorg[0], fsm4);
    for (; u < nunits; u += gridDim.x) {
        const int un = u + gridDim.x;
        __syncthreads();  // every thread is done with the previous unit (its slot and buffer)
        if (tid == 0 && un < nunits) {
            find_tile_cached(I, SHAPE_SWEEP, un >> 1, tcache, sdb[cur ^ 1], s_localb[cur ^ 1]);
            sorg[cur ^ 1] = finish_origin(sdb[cur ^ 1], s_localb[cur ^ 1], un & 1);
        }
        __syncthreads();
        if (un < nunits) finish_stage<r>(sdb[cur ^ 1], sorg[cur ^ 1], fsm4 + (cur ^ 1) * ROWS * CP);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();  // this unit's region has landed
        const ImgDesc &sd = sdb[cur];
        const float4 *sin_ = fsm4 + cur * ROWS * CP;
        const int w = sd.w, h = sd.h, pitch = sd.pitch;
        const int x0 = sorg[cur].x, y0 = sorg[cur].y;
        if (y0 < h) {  // (the lower half of a tile on the last rows may lie below the image)
            // row pass: task e = row e % ROWS, columns 4 (e / ROWS) .. + 3 (one
            // read of the 4 + 2r pixels they share); consecutive lanes take
            // consecutive rows of one column group
            for (int e = tid; e < ROWS * (FX / 4); e += FNT_T) {
                const int g = e / ROWS, ry = e - g * ROWS;
                const float4 *src = sin_ + ry * CP + 4 * g;
                float3 v[4 + 2 * r];
#pragma unroll
                for (int k = 0; k < 4 + 2 * r; ++k) {
                    const float4 t4 = src[k];
                    v[k] = make_float3(t4.x, t4.y, t4.z);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int k = 0; k <= 2 * r; ++k) {
                        a.x = fmaf(wr[k], v[j + k].x, a.x);
                        a.y = fmaf(wr[k], v[j + k].y, a.y);
                        a.z = fmaf(wr[k], v[j + k].z, a.z);
                    }
                    srow[ry * FSR + 4 * g + j] = a;
                }
            }
        }
        __syncthreads();
        if (y0 < h) {
            // column pass: thread = column tid % 32, rows 4 (tid / 32) .. + 3
            const int tx = tid & (FX - 1), ty0 = (tid >> 5) * 4;
            const int gx = x0 + tx;
            float4 win[4 + 2 * r];
#pragma unroll
            for (int q = 0; q < 4 + 2 * r; ++q) win[q] = srow[(ty0 + q) * FSR + tx];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gy = y0 + ty0 + j;
                float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
                for (int k = 0; k <= 2 * r; ++k) {
                    a = fmaf(wr[k], win[j + k].x, a);
                    b = fmaf(wr[k], win[j + k].y, b);
                    d = fmaf(wr[k], win[j + k].z, d);
                }
                if (gx >= w || gy >= h) continue;
                const float m = 0.5f * (a + d), q = 0.5f * (a - d);
                const float det = det2_sym(a, b, d);
                // rr = |(q, b)| and the rotation (cos 2t, sin 2t) = (q, b) / rr: by
                // the fast reciprocal square root (within 2 ulp) where rr^2 is a
                // normal number far from overflow, else by hypot and division
                const float rr2 = fmaf(q, q, b * b);
                float rr, c2 = 1.0f, s2 = 0.0f;
                if (rr2 > 1e-30f && rr2 < 1e30f) {
                    const float inv_rr = rsqrtf(rr2);
                    rr = rr2 * inv_rr;
                    c2 = q * inv_rr;
                    s2 = b * inv_rr;
                } else {
                    rr = hypotf(q, b);
                    if (rr > 0.0f) {
                        const float inv_rr = 1.0f / rr;
                        c2 = q * inv_rr;
                        s2 = b * inv_rr;
                    }
                }
                // the eigenvalue of smaller magnitude as det / (the larger one):
                // a fast division unless the divisor is tiny
                float nu1, nu2;
                if (m > 0.0f) {
                    nu1 = m + rr;
                    nu2 = nu1 > 1e-30f ? __fdividef(det, nu1) : det / nu1;
                } else if (m < 0.0f) {
                    nu2 = m - rr;
                    nu1 = nu2 < -1e-30f ? __fdividef(det, nu2) : det / nu2;
                } else {
                    nu1 = rr;
                    nu2 = -rr;
                }
                const float mu1 = pm_mu(nu1, inv_lambda, mode), mu2 = pm_mu(nu2, inv_lambda, mode);
                if (soa) {  // the FED coefficient planes
                    float *tp = reinterpret_cast<float *>(sd.tensor) + (size_t)gy * pitch + gx;
                    const size_t P = fed_coef_plane(h, pitch);
                    const float qq = 0.25f * (mu1 - mu2);
                    tp[0] = 0.5f * (mu1 + mu2);
                    tp[P] = qq * c2;
                    tp[2 * P] = qq * s2;
                } else {
                    sd.tensor[(size_t)gy * pitch + gx] = make_float4(c2, s2, mu1, mu2);
                }
            }
        }
        cur ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int r>
int launch_finish(const HostBatch &B, const RhoTaps &rt, const fd4_params &p, cudaStream_t st)
{
    static int attr_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    constexpr size_t smem = finish_smem_bytes<r>();
    if (attr_dev != dev) {
        if (cudaFuncSetAttribute(k_tensor_finish<r>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 1;
        attr_dev = dev;
    }
    Imgs I = B.I;
    I.tiles = B.tiles[SHAPE_SWEEP];
    const int grid = persistent_grid((const void *)k_tensor_finish<r>, FNT_T, smem, 2 * I.tiles);
    k_tensor_finish<r><<<grid, FNT_T, smem, st>>>(I, rt, p.lambda, p.mode, B.fed_soa ? 1 : 0);
    return 0;
}

// Opts the sweep kernel into the dynamic shared memory a launch needs.
int set_sweep_smem(size_t bytes)
{
    static size_t done = 0;
    static int done_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (done_dev != dev) {
        done = 0;
        done_dev = dev;
    }
    if (bytes <= done) return 0;
    if (cudaFuncSetAttribute(k_scale_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return 1;
    done = bytes;
    return 0;
}

// Packs the taps of scales [s0, s0 + K) of the set into *t.
int pack_taps(const float *h_sigmas, int n_sigma, int s0, int K, double gamma, SweepTaps *t)
{
    t->K = K;
    t->K_total = n_sigma;
    t->s0 = s0;
    t->Rmax = 0;
    int off = 0;
    for (int s = 0; s < K; ++s) {
        GaussTaps g;
        if (gauss_taps(h_sigmas[s0 + s], &g) != FD4_OK) return 1;
        const int R = (g.r + 3) / 4 * 4, L = 2 * R + 4;
        if (off + 3 * L > kSweepFloats) return 1;
        t->R[s] = R;
        t->off[s] = off;
        t->scale4[s] = (float)pow((double)h_sigmas[s0 + s], 4.0 * gamma);
        if (R > t->Rmax) t->Rmax = R;
        const float *src[3] = {g.w0, g.w1, g.w2};
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < L; ++i) {
                const int o = i - R;  // tap offset
                t->w[off + k * L + i] = (o >= -g.r && o <= g.r) ? src[k][o + g.r] : 0.0f;
            }
        off += 3 * L;
    }
    t->wfloats = off;
    return 0;
}

}  // namespace

template <int r>
static int set_finish_smem()
{
    return cudaFuncSetAttribute(k_tensor_finish<r>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)finish_smem_bytes<r>()) != cudaSuccess;
}

int prepare_scale_kernels()
{
    return set_sweep_smem(sweep_smem_bytes(kMaxRadius, kSweepFloats)) || set_finish_smem<1>() ||
           set_finish_smem<2>() || set_finish_smem<3>() || set_finish_smem<4>() || set_finish_smem<5>() ||
           set_finish_smem<6>() || set_finish_smem<7>() || set_finish_smem<8>() || prepare_tensor_kernels();
}

// Selection planes by the multi-scale tile sweep over B's tile list.
static int sweep_launch(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p, cudaStream_t st)
{
    thread_local static SweepTaps taps;  // 25 KB: kept off the stack
    Imgs I = B.I;
    I.tiles = B.tiles[SHAPE_SWEEP];
    const float inv2b2 = (float)(1.0 / (2.0 * (double)p.beta * p.beta));
    for (int s0 = 0; s0 < n_sigma; s0 += kMaxSweep) {
        const int K = n_sigma - s0 < kMaxSweep ? n_sigma - s0 : kMaxSweep;
        if (pack_taps(h_sigmas, n_sigma, s0, K, p.gamma, &taps)) return 1;
        const size_t smem = sweep_smem_bytes(taps.Rmax, taps.wfloats);
        if (set_sweep_smem(smem)) return 1;
        const int grid = persistent_grid((const void *)k_scale_sweep, NT, smem, I.tiles);
        k_scale_sweep<<<grid, NT, smem, st>>>(I, taps, inv2b2, p.mode);
    }
    return cudaGetLastError() != cudaSuccess;
}

int launch_select_batch(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                        cudaStream_t st)
{
    if (cudaMemsetAsync(B.max_s2, 0, sizeof(unsigned) * (size_t)B.n_max_s2, st) != cudaSuccess) return 1;
    // selection planes: the per-scale strip kernels (fd4_tensor.cu) on whole
    // images, the multi-scale tile sweep (same sums, same order) on a list of
    // tiles (I.list), which the strips cannot walk
    if (B.I.list) {
        if (sweep_launch(B, h_sigmas, n_sigma, p, st)) return 1;
    } else if (launch_select_strips(B, h_sigmas, n_sigma, p, st)) {
        return 1;
    }
    Imgs I = B.I;
    I.tiles = B.tiles[SHAPE_SWEEP];
    const int grid = persistent_grid((const void *)k_select_argmax, 256, 0, I.tiles);
    k_select_argmax<<<grid, 256, 0, st>>>(I, n_sigma, p.c);
    return cudaGetLastError() != cudaSuccess;
}

int launch_tensor_batch(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                        cudaStream_t st)
{
    // N at the selected scales: the per-scale strip kernels (fd4_tensor.cu)
    if (launch_tensor_strips(B, h_sigmas, n_sigma, p, st)) return 1;
    RhoTaps rt;
    if (rho_taps(p.rho, &rt) != FD4_OK) return 1;
    int rc = 1;
    switch (rt.r) {
    case 1: rc = launch_finish<1>(B, rt, p, st); break;
    case 2: rc = launch_finish<2>(B, rt, p, st); break;
    case 3: rc = launch_finish<3>(B, rt, p, st); break;
    case 4: rc = launch_finish<4>(B, rt, p, st); break;
    case 5: rc = launch_finish<5>(B, rt, p, st); break;
    case 6: rc = launch_finish<6>(B, rt, p, st); break;
    case 7: rc = launch_finish<7>(B, rt, p, st); break;
    case 8: rc = launch_finish<8>(B, rt, p, st); break;
    default: rc = 1;
    }
    return rc || cudaGetLastError() != cudaSuccess;
}

// Plain selection on a subset of the 32 x 64 sweep tiles of one image (device
// list of *count tiles): selection planes, the image's max S^2 over those
// tiles, and the argmax written into d.idx on them only.
int launch_select_tiles(const ImgDesc &d, const int *list, const int *count, const float *h_sigmas, int n_sigma,
                        const fd4_params &p, cudaStream_t st)
{
    HostBatch B = single_batch(d);
    B.I.list = list;
    B.I.count = count;
    return launch_select_batch(B, h_sigmas, n_sigma, p, st);
}

// Single-image stages: workspace [header | planes], descriptor passed inline.
int launch_select(const float *d_img, int w, int h, int pitch, const float *h_sigmas, int n_sigma,
                  const fd4_params &p, uint8_t *d_idx, float *d_vmax, char *ws, cudaStream_t st)
{
    WsHeader *hdr = (WsHeader *)ws;
    const size_t pb = plane_bytes(h, pitch, 4);
    ImgDesc d{};
    d.in = d_img;
    d.vp = (float *)(ws + kHeaderBytes);
    d.s2 = (float *)(ws + kHeaderBytes + (size_t)n_sigma * pb);
    d.plane = pb / 4;
    d.idx = d_idx;
    d.vmax = d_vmax;
    d.max_s2 = &hdr->max_s2;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    return launch_select_batch(single_batch(d), h_sigmas, n_sigma, p, st);
}

int launch_tensor(const float *d_u, int w, int h, int pitch, const uint8_t *d_idx, const float *h_sigmas,
                  int n_sigma, const fd4_params &p, float *d_tensor, char *ws, cudaStream_t st)
{
    ImgDesc d{};
    d.u = const_cast<float *>(d_u);  // read only by the tensor build
    d.nfield = (float4 *)(ws + kHeaderBytes);
    d.cmask = (uint32_t *)(ws + kHeaderBytes + plane_bytes(h, pitch, 16));
    d.tensor = (float4 *)d_tensor;
    d.idx = const_cast<uint8_t *>(d_idx);
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    return launch_tensor_batch(single_batch(d), h_sigmas, n_sigma, p, st);
}

static thread_local int g_grid_divisor = 1;
void set_grid_divisor(int d) { g_grid_divisor = d > 0 ? d : 1; }

int persistent_grid(const void *kernel, int threads, size_t smem, int tiles)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 152;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    long long g = (long long)per_sm * sms / g_grid_divisor;
    if (g < 1) g = 1;
    return (int)(tiles < g ? (tiles > 0 ? tiles : 1) : g);
}

}  // namespace fd4
