// FED cycles of the fourth-order anisotropic diffusion (Sec. 3.4 Eq. 17,
// Sec. 3.5 Eq. 21): u <- u - tau_i L^T D L u, n times with D frozen.
//
// The launcher runs one of three kernels, as the schedule says: the
// TMA-staged quad kernel of fd4_fed_tma.cu (2 or 4 steps per launch, natural
// boundary: the default), the scalar fused kernel below (3 steps per launch,
// or the periodic boundary), or one launch per explicit step (k_fed_step).
//
// k_fed_step: one explicit step per launch.  A block stages a 32 x 8 tile of u with a
// 2-pixel halo in shared memory, evaluates T = M D M L u on the tile plus a
// 1-pixel ring (M masks the derivative rows that do not exist under the
// natural boundary), and applies L^T.  Per pixel and step the algorithmic
// HBM traffic is 24 bytes (u read, float4 tensor read, u write); the halo
// re-reads hit L2.
#include "fd4_internal.h"
#include "fd4_quad.cuh"

namespace fd4 {
namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__global__ void __launch_bounds__(BX *BY) k_fed_step(Imgs I, float tau, int parity, int periodic)
{
    __shared__ float su[BY + 4][BX + 4];
    __shared__ float sxx[BY + 2][BX + 2], sxy[BY + 2][BX + 2], syy[BY + 2][BX + 2];
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    __shared__ TileCache tcache;
    if (threadIdx.x == 0) tc_reset(tcache);
    const int tid = threadIdx.y * BX + threadIdx.x;
    for (int t = blockIdx.x; t < I.tiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) find_tile_cached(I, SHAPE_SMALL, t, tcache, sd, s_local);
        __syncthreads();
        const int w = sd.w, h = sd.h, pitch = sd.pitch;
        const float *uin = parity ? sd.tmp : sd.u;
        float *uout = parity ? sd.u : sd.tmp;
        const float4 *ten = sd.tensor;
        const int tiles_x = (w + BX - 1) / BX;
        const int x0 = (s_local % tiles_x) * BX, y0 = (s_local / tiles_x) * BY;

        for (int i = tid; i < (BY + 4) * (BX + 4); i += BX * BY) {
            const int ry = i / (BX + 4), rx = i - ry * (BX + 4);
            int gx = x0 - 2 + rx, gy = y0 - 2 + ry;
            float v = 0.0f;
            if (periodic) {
                v = uin[(size_t)wrap(gy, h) * pitch + wrap(gx, w)];
            } else if (gx >= 0 && gx < w && gy >= 0 && gy < h) {
                v = uin[(size_t)gy * pitch + gx];
            }
            su[ry][rx] = v;
        }
        __syncthreads();

        for (int i = tid; i < (BY + 2) * (BX + 2); i += BX * BY) {
            const int ry = i / (BX + 2), rx = i - ry * (BX + 2);
            int px = x0 - 1 + rx, py = y0 - 1 + ry;
            float Txx = 0.0f, Txy = 0.0f, Tyy = 0.0f;
            bool in = true, vx = true, vy = true;
            if (periodic) {
                px = wrap(px, w);
                py = wrap(py, h);
            } else {
                in = px >= 0 && px < w && py >= 0 && py < h;
                vx = px >= 1 && px <= w - 2;
                vy = py >= 1 && py <= h - 2;
            }
            if (in && (vx || vy)) {
                const float c = su[ry + 1][rx + 1];
                const float hxx = vx ? su[ry + 1][rx] - 2.0f * c + su[ry + 1][rx + 2] : 0.0f;
                const float hyy = vy ? su[ry][rx + 1] - 2.0f * c + su[ry + 2][rx + 1] : 0.0f;
                const float hxy =
                    (vx && vy) ? 0.25f * (su[ry][rx] + su[ry + 2][rx + 2] - su[ry + 2][rx] - su[ry][rx + 2]) : 0.0f;
                const float4 tt = __ldg(ten + (size_t)py * pitch + px);  // (cos 2t, sin 2t, mu1, mu2)
                // D : h in the eigenframe of e1 = (cos t, sin t), e2 = (-sin t, cos t)
                const float sh = 0.5f * (hxx + hyy), dh = 0.5f * (hxx - hyy);
                const float h11 = sh + tt.x * dh + tt.y * hxy;
                const float h22 = sh - tt.x * dh - tt.y * hxy;
                const float h12 = tt.x * hxy - tt.y * dh;
                const float t11 = tt.z * h11, t22 = tt.w * h22, t12 = 0.5f * (tt.z + tt.w) * h12;
                const float st = 0.5f * (t11 + t22), dt = 0.5f * (t11 - t22);
                Txx = vx ? st + tt.x * dt - tt.y * t12 : 0.0f;
                Tyy = vy ? st - tt.x * dt + tt.y * t12 : 0.0f;
                Txy = (vx && vy) ? tt.y * dt + tt.x * t12 : 0.0f;
            }
            sxx[ry][rx] = Txx;
            sxy[ry][rx] = Txy;
            syy[ry][rx] = Tyy;
        }
        __syncthreads();

        const int tx = threadIdx.x, ty = threadIdx.y;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= w || gy >= h) continue;
        const float div = (sxx[ty + 1][tx] - 2.0f * sxx[ty + 1][tx + 1] + sxx[ty + 1][tx + 2]) +
                          (syy[ty][tx + 1] - 2.0f * syy[ty + 1][tx + 1] + syy[ty + 2][tx + 1]) +
                          0.5f * (sxy[ty + 2][tx + 2] + sxy[ty][tx] - sxy[ty][tx + 2] - sxy[ty + 2][tx]);
        uout[(size_t)gy * pitch + gx] = su[ty + 2][tx + 2] - tau * div;
    }
}

// Copies each image's input into its filter state (skipped where they coincide).
__global__ void __launch_bounds__(256) k_copy_in(Imgs I)
{
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    __shared__ TileCache tcache;
    if (threadIdx.x == 0) tc_reset(tcache);
    const int tid = threadIdx.x;
    for (int t = blockIdx.x; t < I.tiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) find_tile_cached(I, SHAPE_SMALL, t, tcache, sd, s_local);
        __syncthreads();
        if (sd.in == sd.u) continue;
        const int tiles_x = (sd.w + 31) / 32;
        const int x = (s_local % tiles_x) * 32 + (tid & 31), y = (s_local / tiles_x) * 8 + (tid >> 5);
        if (x < sd.w && y < sd.h) sd.u[(size_t)y * sd.pitch + x] = sd.in[(size_t)y * sd.pitch + x];
    }
}

// Writes a chunk of batch descriptors (passed as kernel parameters) to the
// device table, so the upload is an ordinary kernel node in a CUDA graph.
constexpr int kDescChunk = 128;
struct DescChunk {
    int first, n;
    ImgDesc d[kDescChunk];
};
__global__ void k_put_descs(DescChunk c, ImgDesc *table)
{
    const int i = threadIdx.x;
    if (i < c.n) table[c.first + i] = c.d[i];
}

// Copies the FED ping-pong plane back into the image (odd number of launches).
__global__ void __launch_bounds__(256) k_copy_back(Imgs I)
{
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    __shared__ TileCache tcache;
    if (threadIdx.x == 0) tc_reset(tcache);
    const int tid = threadIdx.x;
    for (int t = blockIdx.x; t < I.tiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) find_tile_cached(I, SHAPE_SMALL, t, tcache, sd, s_local);
        __syncthreads();
        const int tiles_x = (sd.w + 31) / 32;
        const int x = (s_local % tiles_x) * 32 + (tid & 31), y = (s_local / tiles_x) * 8 + (tid >> 5);
        if (x < sd.w && y < sd.h) sd.u[(size_t)y * sd.pitch + x] = sd.tmp[(size_t)y * sd.pitch + x];
    }
}


// ---------------------------------------------------------------------------
// Fused variant: S explicit steps per launch (overlapped temporal blocking).
// A block stages a RX x RY = 64 x 32 region of u (the output tile plus a halo
// of H = 2S pixels) in shared memory and advances it S steps there; step l
// computes T on the region shrunk by 2l+1 and u on the region shrunk by 2l+2,
// so after S steps the (64-4S) x (32-4S) interior is exact and is written
// back.  Each thread owns a column segment of 4 pixels for the whole launch:
// it loads their tensor values once into registers (D is frozen over the
// cycle) and slides 3-row register windows over u and T, so a pixel-step
// costs about 4.5 shared loads for T and 7.5 for the update instead of 9 and 10.
// HBM traffic per pixel-step falls from 24 B to about 24/S B plus halo.

constexpr int FRX = 64, FRY = 32, FV = 4, FNT = (FRX / 32) * (FRY / FV) * 32;  // 512 threads
constexpr size_t kFusedSmem = 4 * sizeof(float) * FRX * FRY;                  // 32 KB


// The S steps of one staged region.  INTERIOR: the region lies inside the
// image (natural boundary), so every derivative row exists and no mask or
// bounds test is needed; otherwise per-pixel masks follow the natural (or
// periodic) boundary.  rowbits: bit j = pixel row j of the segment is inside
// the image, bit 8 + j = its Lyy row exists.
template <bool INTERIOR>
__device__ __forceinline__ void fused_steps(float (*su)[FRX], float (*sxx)[FRX], float (*sxy)[FRX],
                                            float (*syy)[FRX], const float *stau, int nsteps, int rx, int ry0,
                                            const float4 (&tv)[FV], bool in_x, bool vx, unsigned rowbits)
{
    const int xl = rx > 0 ? rx - 1 : 0, xr = rx < FRX - 1 ? rx + 1 : FRX - 1;
    for (int l = 0; l < nsteps; ++l) {
        // T = M D M L u where the region shrunk by 2l+1 holds valid data
        const int lo_t = 2 * l + 1;
        const bool col_t = rx >= lo_t && rx < FRX - lo_t;
        {
            const int rm = ry0 > 0 ? ry0 - 1 : 0;
            float aL = su[rm][xl], aC = su[rm][rx], aR = su[rm][xr];
            float bL = su[ry0][xl], bC = su[ry0][rx], bR = su[ry0][xr];
#pragma unroll
            for (int j = 0; j < FV; ++j) {
                const int ry = ry0 + j;
                const int rp = ry + 1 < FRY ? ry + 1 : FRY - 1;
                const float cL = su[rp][xl], cC = su[rp][rx], cR = su[rp][xr];
                if (col_t && ry >= lo_t && ry < FRY - lo_t) {
                    const bool in = INTERIOR || (in_x && ((rowbits >> j) & 1u));
                    const bool vy = INTERIOR || ((rowbits >> (8 + j)) & 1u);
                    const bool vxx = INTERIOR || vx;
                    float Txx = 0.0f, Txy = 0.0f, Tyy = 0.0f;
                    if (in && (vxx || vy)) {
                        const float hxx = vxx ? bL - 2.0f * bC + bR : 0.0f;
                        const float hyy = vy ? aC - 2.0f * bC + cC : 0.0f;
                        const float hxy = (vxx && vy) ? 0.25f * (aL + cR - cL - aR) : 0.0f;
                        const float4 tt = tv[j];
                        const float sh = 0.5f * (hxx + hyy), dh = 0.5f * (hxx - hyy);
                        const float h11 = sh + tt.x * dh + tt.y * hxy;
                        const float h22 = sh - tt.x * dh - tt.y * hxy;
                        const float h12 = tt.x * hxy - tt.y * dh;
                        const float t11 = tt.z * h11, t22 = tt.w * h22, t12 = 0.5f * (tt.z + tt.w) * h12;
                        const float st = 0.5f * (t11 + t22), dt = 0.5f * (t11 - t22);
                        Txx = vxx ? st + tt.x * dt - tt.y * t12 : 0.0f;
                        Tyy = vy ? st - tt.x * dt + tt.y * t12 : 0.0f;
                        Txy = (vxx && vy) ? tt.y * dt + tt.x * t12 : 0.0f;
                    }
                    sxx[ry][rx] = Txx;
                    sxy[ry][rx] = Txy;
                    syy[ry][rx] = Tyy;
                }
                aL = bL; aC = bC; aR = bR;
                bL = cL; bC = cC; bR = cR;
            }
        }
        __syncthreads();
        // u -= tau (Lxx' Txx + Lyy' Tyy + 2 Lxy' Txy) on the region shrunk by 2l+2
        const int lo_u = 2 * l + 2;
        if (rx >= lo_u && rx < FRX - lo_u) {
            const float tau = stau[l];
            const int rm = ry0 > 0 ? ry0 - 1 : 0;
            float yA = syy[rm][rx], yB = syy[ry0][rx];
            float dLA = sxy[rm][xl], dRA = sxy[rm][xr], dLB = sxy[ry0][xl], dRB = sxy[ry0][xr];
#pragma unroll
            for (int j = 0; j < FV; ++j) {
                const int ry = ry0 + j;
                const int rp = ry + 1 < FRY ? ry + 1 : FRY - 1;
                const float yC = syy[rp][rx];
                const float dLC = sxy[rp][xl], dRC = sxy[rp][xr];
                if (ry >= lo_u && ry < FRY - lo_u) {
                    const bool in = INTERIOR || (in_x && ((rowbits >> j) & 1u));
                    if (in) {
                        const float div = (sxx[ry][xl] - 2.0f * sxx[ry][rx] + sxx[ry][xr]) +
                                          (yA - 2.0f * yB + yC) + 0.5f * (dRC + dLA - dRA - dLC);
                        su[ry][rx] -= tau * div;
                    }
                }
                yA = yB; yB = yC;
                dLA = dLB; dRA = dRB;
                dLB = dLC; dRB = dRC;
            }
        }
        __syncthreads();
    }
}

template <int S>
__global__ void __launch_bounds__(FNT, 2) k_fed_fused(Imgs I, StepTaus taus, int parity, int periodic)
{
    constexpr int H = 2 * S, TXo = FRX - 2 * H, TYo = FRY - 2 * H;
    extern __shared__ float fsm[];
    float (*su)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm);
    float (*sxx)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm + FRX * FRY);
    float (*sxy)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm + 2 * FRX * FRY);
    float (*syy)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm + 3 * FRX * FRY);
    __shared__ float stau[8];
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) stau[i] = taus.t[i];
    }
    // this thread's column segment of the staged region
    const int rx = (warp % (FRX / 32)) * 32 + lane, ry0 = (warp / (FRX / 32)) * FV;

    for (int t = blockIdx.x; t < I.tiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) find_tile(I, S, t, sd, s_local);
        __syncthreads();
        const int w = sd.w, h = sd.h, pitch = sd.pitch;
        const float *uin = parity ? sd.tmp : sd.u;
        float *uout = parity ? sd.u : sd.tmp;
        const float4 *ten = sd.tensor;
        const int tiles_x = (w + TXo - 1) / TXo;
        const int gx0 = (s_local % tiles_x) * TXo - H, gy0 = (s_local / tiles_x) * TYo - H;
        const bool interior = !periodic && gx0 >= 0 && gy0 >= 0 && gx0 + FRX <= w && gy0 + FRY <= h;

        if (interior) {
            for (int i = tid; i < FRX * FRY; i += FNT) {
                const int ry = i / FRX, rxx = i - ry * FRX;
                su[ry][rxx] = uin[(size_t)(gy0 + ry) * pitch + gx0 + rxx];
            }
        } else {
            for (int i = tid; i < FRX * FRY; i += FNT) {
                const int ry = i / FRX, rxx = i - ry * FRX;
                const int gx = gx0 + rxx, gy = gy0 + ry;
                float v = 0.0f;
                if (periodic) v = uin[(size_t)wrap(gy, h) * pitch + wrap(gx, w)];
                else if (gx >= 0 && gx < w && gy >= 0 && gy < h) v = uin[(size_t)gy * pitch + gx];
                su[ry][rxx] = v;
            }
        }

        // the tensor values of this thread's pixels (D is frozen over the cycle)
        const int gx = gx0 + rx;
        const int pgx = periodic ? wrap(gx, w) : gx;
        const bool in_x = periodic || (gx >= 0 && gx < w);
        const bool vx = periodic || (gx >= 1 && gx <= w - 2);
        unsigned rowbits = 0u;
        float4 tv[FV];
#pragma unroll
        for (int j = 0; j < FV; ++j) {
            const int gy = gy0 + ry0 + j;
            const bool iny = periodic || (gy >= 0 && gy < h);
            const bool vy = periodic || (gy >= 1 && gy <= h - 2);
            rowbits |= (iny ? 1u : 0u) << j;
            rowbits |= (vy ? 1u : 0u) << (8 + j);
            tv[j] = (in_x && iny) ? __ldg(ten + (size_t)(periodic ? wrap(gy, h) : gy) * pitch + pgx)
                                  : make_float4(1.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();

        if (interior) fused_steps<true>(su, sxx, sxy, syy, stau, taus.n, rx, ry0, tv, in_x, vx, rowbits);
        else fused_steps<false>(su, sxx, sxy, syy, stau, taus.n, rx, ry0, tv, in_x, vx, rowbits);

        for (int i = tid; i < TXo * TYo; i += FNT) {
            const int ty = i / TXo, tx = i - ty * TXo;
            const int ox = gx0 + H + tx, oy = gy0 + H + ty;
            if (ox < w && oy < h) uout[(size_t)oy * pitch + ox] = su[H + ty][H + tx];
        }
    }
}

}  // namespace

template <int S>
static int set_fused_smem()
{
    static int attr_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (attr_dev != dev) {
        if (cudaFuncSetAttribute(k_fed_fused<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem) !=
            cudaSuccess)
            return 1;
        attr_dev = dev;
    }
    return 0;
}

int prepare_fed_kernels()
{
    return set_fused_smem<2>() || set_fused_smem<3>() || set_fused_smem<4>() || prepare_tma_kernels();
}

template <int S>
static int launch_fused(Imgs I, const double *tau, int n, int parity, int periodic, cudaStream_t st)
{
    if (set_fused_smem<S>()) return 1;
    StepTaus t{};
    t.n = n;
    for (int i = 0; i < n; ++i) t.t[i] = (float)tau[i];
    const int grid = persistent_grid((const void *)k_fed_fused<S>, FNT, kFusedSmem, I.tiles);
    k_fed_fused<S><<<grid, FNT, kFusedSmem, st>>>(I, t, parity, periodic);
    return 0;
}

FedSched resolve_sched(const fd4_params &p)
{
    FedSched s;
    s.steps = p.fed_steps_per_launch > 0 ? p.fed_steps_per_launch : kDefaultSched.steps;
    s.rows = p.fed_tile_rows > 0 ? p.fed_tile_rows : kDefaultSched.rows;
    s.quads = p.fed_quads_per_thread > 0 ? p.fed_quads_per_thread : kDefaultSched.quads;
    return s;
}

int launch_copy_back_batch(const HostBatch &B, cudaStream_t st)
{
    Imgs I = B.I;
    I.tiles = B.tiles[SHAPE_SMALL];
    const int grid = persistent_grid((const void *)k_copy_back, 256, 0, I.tiles);
    k_copy_back<<<grid, 256, 0, st>>>(I);
    return cudaGetLastError() != cudaSuccess;
}

int launch_fed_batch(const HostBatch &B, const double *h_tau, int n, int boundary, const FedSched &sch,
                     cudaStream_t st, int *end_parity)
{
    const int periodic = boundary == FD4_BC_PERIODIC;
    int S = sch.steps;
    if (S < 1 || S > 4) S = kDefaultSched.steps;
    // the FED coefficient planes are read by the TMA kernel only
    if (B.fed_soa && (periodic || S == 1 || S == 3)) return 1;
    int parity = 0;
    if (S == 1) {
        Imgs I = B.I;
        I.tiles = B.tiles[SHAPE_SMALL];
        const int grid = persistent_grid((const void *)k_fed_step, BX * BY, 0, I.tiles);
        for (int i = 0; i < n; ++i) {
            k_fed_step<<<grid, dim3(BX, BY), 0, st>>>(I, (float)h_tau[i], parity, periodic);
            parity ^= 1;
        }
    } else {
        Imgs I = B.I;
        I.tiles = B.tiles[S];
        for (int i = 0; i < n; i += S) {
            const int k = n - i < S ? n - i : S;
            int rc;
            // the TMA-staged quad kernel for 2 and 4 steps under the natural
            // boundary; the scalar fused kernel for 3 steps and the periodic boundary
            if (!periodic && S != 3)
                rc = S == 2 ? launch_fed_tma<2>(B, h_tau + i, k, parity, sch, st)
                            : launch_fed_tma<4>(B, h_tau + i, k, parity, sch, st);
            else
                rc = S == 2 ? launch_fused<2>(I, h_tau + i, k, parity, periodic, st)
                   : S == 3 ? launch_fused<3>(I, h_tau + i, k, parity, periodic, st)
                            : launch_fused<4>(I, h_tau + i, k, parity, periodic, st);
            if (rc) return 1;
            parity ^= 1;
        }
    }
    if (end_parity) *end_parity = parity;
    else if (parity && launch_copy_back_batch(B, st)) return 1;  // the last launch wrote the ping-pong plane
    return cudaGetLastError() != cudaSuccess;
}

int launch_copy_in_batch(const HostBatch &B, cudaStream_t st)
{
    Imgs I = B.I;
    I.tiles = B.tiles[SHAPE_SMALL];
    const int grid = persistent_grid((const void *)k_copy_in, 256, 0, I.tiles);
    k_copy_in<<<grid, 256, 0, st>>>(I);
    return cudaGetLastError() != cudaSuccess;
}

int launch_put_descs(const ImgDesc *h_descs, int n, ImgDesc *d_table, cudaStream_t st)
{
    thread_local static DescChunk c;  // ~15 KB: kept off the stack
    for (int first = 0; first < n; first += kDescChunk) {
        c.first = first;
        c.n = n - first < kDescChunk ? n - first : kDescChunk;
        for (int i = 0; i < c.n; ++i) c.d[i] = h_descs[first + i];
        k_put_descs<<<1, kDescChunk, 0, st>>>(c, d_table);
    }
    return cudaGetLastError() != cudaSuccess;
}

int launch_fed_cycle(float *d_u, int w, int h, int pitch, const float *d_tensor, const double *h_tau, int n,
                     int boundary, const FedSched &sch, char *ws, cudaStream_t st)
{
    ImgDesc d{};
    d.u = d_u;
    d.tmp = (float *)(ws + kHeaderBytes);
    d.tensor = (float4 *)d_tensor;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    return launch_fed_batch(single_batch(d), h_tau, n, boundary, sch, st);
}

}  // namespace fd4
