// FED cycles of the fourth-order anisotropic diffusion (Sec. 3.4 Eq. 17,
// Sec. 3.5 Eq. 21): u <- u - tau_i L^T D L u, n times with D frozen.
//
// One explicit step per launch.  A block stages a 32 x 8 tile of u with a
// 2-pixel halo in shared memory, evaluates T = M D M L u on the tile plus a
// 1-pixel ring (M masks the derivative rows that do not exist under the
// natural boundary), and applies L^T.  Per pixel and step the algorithmic
// HBM traffic is 24 bytes (u read, float4 tensor read, u write); the halo
// re-reads hit L2.
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

}  // namespace

int launch_fed_cycle(float *d_u, int w, int h, int pitch, const float *d_tensor, const double *h_tau, int n,
                     int boundary, char *ws, cudaStream_t st)
{
    float *tmp = (float *)(ws + kHeaderBytes);
    const dim3 grid((w + BX - 1) / BX, (h + BY - 1) / BY), block(BX, BY);
    const float4 *ten = (const float4 *)d_tensor;
    float *a = d_u, *b = tmp;
    for (int i = 0; i < n; ++i) {
        k_fed_step<<<grid, block, 0, st>>>(a, b, ten, w, h, pitch, (float)h_tau[i], boundary == FD4_BC_PERIODIC);
        float *t = a;
        a = b;
        b = t;
    }
    if (a != d_u) {
        if (cudaMemcpy2DAsync(d_u, (size_t)pitch * 4, a, (size_t)pitch * 4, (size_t)w * 4, (size_t)h,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return 1;
    }
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace fd4
