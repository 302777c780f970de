// FED cycles of the fourth-order anisotropic diffusion (Sec. 3.4 Eq. 17,
// Sec. 3.5 Eq. 21): u <- u - tau_i L^T D L u, n times with D frozen.
//
// One explicit step per launch.  A block stages a 32 x 8 tile of u with a
// 2-pixel halo in shared memory, evaluates T = M D M L u on the tile plus a
// 1-pixel ring (M masks the derivative rows that do not exist under the
// natural boundary), and applies L^T.  Per pixel and step the algorithmic
// HBM traffic is 24 bytes (u read, float4 tensor read, u write); the halo
// re-reads hit L2.
#include <cstdlib>

#include "fd4_internal.h"

namespace fd4 {
namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__global__ void __launch_bounds__(BX *BY) k_fed_step(const float *__restrict__ uin, float *__restrict__ uout,
                                                     const float4 *__restrict__ ten, int w, int h, int pitch,
                                                     float tau, int periodic)
{
    __shared__ float su[BY + 4][BX + 4];
    __shared__ float sxx[BY + 2][BX + 2], sxy[BY + 2][BX + 2], syy[BY + 2][BX + 2];
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int tid = threadIdx.y * BX + threadIdx.x;

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
            const float hxy = (vx && vy) ? 0.25f * (su[ry][rx] + su[ry + 2][rx + 2] - su[ry + 2][rx] - su[ry][rx + 2])
                                         : 0.0f;
            const float4 t = __ldg(ten + (size_t)py * pitch + px);  // (cos 2t, sin 2t, mu1, mu2)
            // D : h in the eigenframe of e1 = (cos t, sin t), e2 = (-sin t, cos t)
            const float sh = 0.5f * (hxx + hyy), dh = 0.5f * (hxx - hyy);
            const float h11 = sh + t.x * dh + t.y * hxy;
            const float h22 = sh - t.x * dh - t.y * hxy;
            const float h12 = t.x * hxy - t.y * dh;
            const float t11 = t.z * h11, t22 = t.w * h22, t12 = 0.5f * (t.z + t.w) * h12;
            const float st = 0.5f * (t11 + t22), dt = 0.5f * (t11 - t22);
            Txx = vx ? st + t.x * dt - t.y * t12 : 0.0f;
            Tyy = vy ? st - t.x * dt + t.y * t12 : 0.0f;
            Txy = (vx && vy) ? t.y * dt + t.x * t12 : 0.0f;
        }
        sxx[ry][rx] = Txx;
        sxy[ry][rx] = Txy;
        syy[ry][rx] = Tyy;
    }
    __syncthreads();

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= w || gy >= h) return;
    const float div = (sxx[ty + 1][tx] - 2.0f * sxx[ty + 1][tx + 1] + sxx[ty + 1][tx + 2]) +
                      (syy[ty][tx + 1] - 2.0f * syy[ty + 1][tx + 1] + syy[ty + 2][tx + 1]) +
                      0.5f * (sxy[ty + 2][tx + 2] + sxy[ty][tx] - sxy[ty][tx + 2] - sxy[ty + 2][tx]);
    uout[(size_t)gy * pitch + gx] = su[ty + 2][tx + 2] - tau * div;
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

struct StepTaus {
    float t[8];
    int n;
};

template <int S>
__global__ void __launch_bounds__(FNT, 2) k_fed_fused(const float *__restrict__ uin, float *__restrict__ uout,
                                                      const float4 *__restrict__ ten, int w, int h, int pitch,
                                                      StepTaus taus, int periodic)
{
    constexpr int H = 2 * S, TXo = FRX - 2 * H, TYo = FRY - 2 * H;
    extern __shared__ float fsm[];
    float (*su)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm);
    float (*sxx)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm + FRX * FRY);
    float (*sxy)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm + 2 * FRX * FRY);
    float (*syy)[FRX] = reinterpret_cast<float (*)[FRX]>(fsm + 3 * FRX * FRY);

    __shared__ float stau[8];
    const int gx0 = blockIdx.x * TXo - H, gy0 = blockIdx.y * TYo - H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 8) stau[tid] = taus.t[tid];

    for (int i = tid; i < FRX * FRY; i += FNT) {
        const int ry = i / FRX, rx = i - ry * FRX;
        const int gx = gx0 + rx, gy = gy0 + ry;
        float v = 0.0f;
        if (periodic) v = uin[(size_t)wrap(gy, h) * pitch + wrap(gx, w)];
        else if (gx >= 0 && gx < w && gy >= 0 && gy < h) v = uin[(size_t)gy * pitch + gx];
        su[ry][rx] = v;
    }

    // this thread's column segment and its pixels' tensor values
    const int rx = (warp % (FRX / 32)) * 32 + lane, ry0 = (warp / (FRX / 32)) * FV;
    const int gx = gx0 + rx;
    const int pgx = periodic ? wrap(gx, w) : gx;
    const bool in_x = periodic || (gx >= 0 && gx < w);
    const bool vx = periodic || (gx >= 1 && gx <= w - 2);
    float4 tv[FV];
#pragma unroll
    for (int j = 0; j < FV; ++j) {
        const int gy = gy0 + ry0 + j;
        const bool in = in_x && (periodic || (gy >= 0 && gy < h));
        tv[j] = in ? __ldg(ten + (size_t)(periodic ? wrap(gy, h) : gy) * pitch + pgx) : make_float4(1.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    const int xl = rx > 0 ? rx - 1 : 0, xr = rx < FRX - 1 ? rx + 1 : FRX - 1;
    for (int l = 0; l < taus.n; ++l) {
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
                    const int gy = gy0 + ry;
                    const bool in = in_x && (periodic || (gy >= 0 && gy < h));
                    const bool vy = periodic || (gy >= 1 && gy <= h - 2);
                    float Txx = 0.0f, Txy = 0.0f, Tyy = 0.0f;
                    if (in && (vx || vy)) {
                        const float hxx = vx ? bL - 2.0f * bC + bR : 0.0f;
                        const float hyy = vy ? aC - 2.0f * bC + cC : 0.0f;
                        const float hxy = (vx && vy) ? 0.25f * (aL + cR - cL - aR) : 0.0f;
                        const float4 t = tv[j];
                        const float sh = 0.5f * (hxx + hyy), dh = 0.5f * (hxx - hyy);
                        const float h11 = sh + t.x * dh + t.y * hxy;
                        const float h22 = sh - t.x * dh - t.y * hxy;
                        const float h12 = t.x * hxy - t.y * dh;
                        const float t11 = t.z * h11, t22 = t.w * h22, t12 = 0.5f * (t.z + t.w) * h12;
                        const float st = 0.5f * (t11 + t22), dt = 0.5f * (t11 - t22);
                        Txx = vx ? st + t.x * dt - t.y * t12 : 0.0f;
                        Tyy = vy ? st - t.x * dt + t.y * t12 : 0.0f;
                        Txy = (vx && vy) ? t.y * dt + t.x * t12 : 0.0f;
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
                    const int gy = gy0 + ry;
                    const bool in = in_x && (periodic || (gy >= 0 && gy < h));
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

    for (int i = tid; i < TXo * TYo; i += FNT) {
        const int ty = i / TXo, tx = i - ty * TXo;
        const int ox = gx0 + H + tx, oy = gy0 + H + ty;
        if (ox < w && oy < h) uout[(size_t)oy * pitch + ox] = su[H + ty][H + tx];
    }
}

}  // namespace

// Steps fused per launch: FD4_FED_FUSE in the environment (0 = one launch per
// step with k_fed_step, 2..4 = k_fed_fused<S>); default 2.
static int fuse_steps()
{
    const char *e = getenv("FD4_FED_FUSE");
    if (!e) return 2;
    const int v = atoi(e);
    return (v == 0 || (v >= 2 && v <= 4)) ? v : 2;
}

template <int S>
static int launch_fused(const float *a, float *b, const float4 *ten, int w, int h, int pitch, const double *tau,
                        int n, int periodic, cudaStream_t st)
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
    constexpr int TXo = FRX - 4 * S, TYo = FRY - 4 * S;
    const dim3 grid((w + TXo - 1) / TXo, (h + TYo - 1) / TYo);
    StepTaus t{};
    t.n = n;
    for (int i = 0; i < n; ++i) t.t[i] = (float)tau[i];
    k_fed_fused<S><<<grid, FNT, kFusedSmem, st>>>(a, b, ten, w, h, pitch, t, periodic);
    return 0;
}

int launch_fed_cycle(float *d_u, int w, int h, int pitch, const float *d_tensor, const double *h_tau, int n,
                     int boundary, char *ws, cudaStream_t st)
{
    float *tmp = (float *)(ws + kHeaderBytes);
    const float4 *ten = (const float4 *)d_tensor;
    const int periodic = boundary == FD4_BC_PERIODIC;
    const int S = fuse_steps();
    float *a = d_u, *b = tmp;
    if (S == 0) {
        const dim3 grid((w + BX - 1) / BX, (h + BY - 1) / BY), block(BX, BY);
        for (int i = 0; i < n; ++i) {
            k_fed_step<<<grid, block, 0, st>>>(a, b, ten, w, h, pitch, (float)h_tau[i], periodic);
            float *t = a;
            a = b;
            b = t;
        }
    } else {
        for (int i = 0; i < n; i += S) {
            const int k = n - i < S ? n - i : S;
            int rc = S == 2 ? launch_fused<2>(a, b, ten, w, h, pitch, h_tau + i, k, periodic, st)
                   : S == 3 ? launch_fused<3>(a, b, ten, w, h, pitch, h_tau + i, k, periodic, st)
                            : launch_fused<4>(a, b, ten, w, h, pitch, h_tau + i, k, periodic, st);
            if (rc) return 1;
            float *t = a;
            a = b;
            b = t;
        }
    }
    if (a != d_u) {
        if (cudaMemcpy2DAsync(d_u, (size_t)pitch * 4, a, (size_t)pitch * 4, (size_t)w * 4, (size_t)h,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return 1;
    }
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace fd4
