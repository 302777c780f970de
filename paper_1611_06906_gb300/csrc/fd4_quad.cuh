// Quad form of one FED step (Sec. 3.4 Eq. 17: u <- u - tau L^T D L u) shared
// by the FED kernels that give each thread a row quad (4 adjacent pixels of one
// row): T = M D M L u with D applied in its eigenframe, then the divergence.
// Horizontal neighbours come from the adjacent lanes (shuffles), vertical ones
// from the shared-memory planes (row stride SW floats).
#pragma once

#include "fd4_internal.h"

namespace fd4 {

// Step sizes of one fused launch (up to 8 steps).
struct StepTaus {
    float t[8];
    int n;
};

// Per pixel of the quad, from the tensor field (cos 2t, sin 2t, mu1, mu2):
// m = mu3 = (mu1 + mu2) / 2, and with q = (mu1 - mu2) / 4: qc = q cos 2t,
// qs = q sin 2t, qs2 = 2 qs.
struct QuadCoef {
    float4 m, qc, qs, qs2;
};

__device__ __forceinline__ void f4_to(const float4 v, float *d)
{
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}

// The quad's 4 values with the left and right neighbours from adjacent lanes.
__device__ __forceinline__ void quad_ext(const float4 m, float (&v)[6])
{
    v[0] = __shfl_up_sync(0xffffffffu, m.w, 1);
    v[1] = m.x; v[2] = m.y; v[3] = m.z; v[4] = m.w;
    v[5] = __shfl_down_sync(0xffffffffu, m.x, 1);
}

// T = M D M L u for the 4 pixels of one quad.  a, b, c: rows y-1, y, y+1 at
// columns x-1 .. x+4.  BOUNDARY: apply the natural-boundary masks (bits 0-3:
// pixel inside, 4-7: Lxx row exists, 8: Lyy row exists for this row).
// D acts on the Hessian H through its eigentensors: with E1, E2 the projectors
// on the eigenvectors, t11 = mu1 h11, t22 = mu2 h22 and t12 = mu3 h12 give
//   T = mu3 H + (mu1 - mu2) / 2 (h11 E1 - h22 E2) = mu3 H + q (z I + tr H R),
// where R = E1 - E2 = [[c, s], [s, -c]] (c = cos 2t, s = sin 2t),
// z = R:H = c (hxx - hyy) + 2 s hxy and q = (mu1 - mu2) / 4.  So
//   Txx = mu3 hxx + Z + qc tr H,  Tyy = mu3 hyy + Z - qc tr H,
//   Txy = mu3 hxy + qs tr H,      Z = qc (hxx - hyy) + 2 qs hxy,
// ten operations for T per pixel on three coefficients (and 2 qs).  The mixed
// derivative shares its column differences a - c between neighbouring pixels.
template <bool BOUNDARY>
__device__ __forceinline__ void quad_T(const float (&a)[6], const float (&b)[6], const float (&c)[6],
                                       const QuadCoef &k, unsigned mask, float4 &Txx, float4 &Txy, float4 &Tyy)
{
    float rxx[4], rxy[4], ryy[4];
    float mm[4], qc[4], qs[4], q2[4];
    f4_to(k.m, mm);
    f4_to(k.qc, qc);
    f4_to(k.qs, qs);
    f4_to(k.qs2, q2);
    float e[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) e[j] = a[j] - c[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float hxx = fmaf(-2.0f, b[i + 1], b[i] + b[i + 2]);
        float hyy = fmaf(-2.0f, b[i + 1], a[i + 1] + c[i + 1]);
        float hxy = 0.25f * (e[i] - e[i + 2]);
        bool vx = true, vy = true, in = true;
        if (BOUNDARY) {
            in = (mask >> i) & 1u;
            vx = (mask >> (4 + i)) & 1u;
            vy = (mask >> 8) & 1u;
            hxx = vx ? hxx : 0.0f;
            hyy = vy ? hyy : 0.0f;
            hxy = (vx && vy) ? hxy : 0.0f;
        }
        const float tr = hxx + hyy, dh = hxx - hyy;
        const float Z = fmaf(qc[i], dh, q2[i] * hxy);  // q z
        float txx = fmaf(mm[i], hxx, fmaf(qc[i], tr, Z));
        float tyy = fmaf(mm[i], hyy, fmaf(-qc[i], tr, Z));
        float txy = fmaf(mm[i], hxy, qs[i] * tr);
        if (BOUNDARY) {
            txx = (in && vx) ? txx : 0.0f;
            tyy = (in && vy) ? tyy : 0.0f;
            txy = (in && vx && vy) ? txy : 0.0f;
        }
        rxx[i] = txx;
        rxy[i] = txy;
        ryy[i] = tyy;
    }
    Txx = make_float4(rxx[0], rxx[1], rxx[2], rxx[3]);
    Txy = make_float4(rxy[0], rxy[1], rxy[2], rxy[3]);
    Tyy = make_float4(ryy[0], ryy[1], ryy[2], ryy[3]);
}

struct NoHook {
    __device__ void operator()() const {}
};

// S steps of one staged region for NQ quads per thread; uo: the quads' u on
// entry, updated in place.  Two block barriers per step: T is complete before
// the update reads it, the update is complete before the next T phase reads u.
// The first T phase reads the staged region (published by the tile's
// barrier); after the last update no barrier is needed before the next tile's.
// hook() runs once, right after the first step's T barrier (every thread is
// then past whatever it read before the call).
template <bool BOUNDARY, int SW, int NQ, class Hook = NoHook>
__device__ __forceinline__ void quad_steps_n(float *su, float *sxy, float *syy, const float *stau, int nsteps,
                                             const int (&off)[NQ], const QuadCoef (&k)[NQ],
                                             const unsigned (&mask)[NQ], float4 (&uo)[NQ],
                                             const Hook &hook = Hook())
{
    for (int l = 0; l < nsteps; ++l) {
        if (l > 0) __syncthreads();
        float4 txx[NQ], tyy[NQ];
#pragma unroll
        for (int qd = 0; qd < NQ; ++qd) {
            float a[6], b[6], c[6];
            quad_ext(*reinterpret_cast<const float4 *>(su + off[qd] - SW), a);
            quad_ext(uo[qd], b);
            quad_ext(*reinterpret_cast<const float4 *>(su + off[qd] + SW), c);
            float4 txy;
            quad_T<BOUNDARY>(a, b, c, k[qd], mask[qd], txx[qd], txy, tyy[qd]);
            *reinterpret_cast<float4 *>(sxy + off[qd]) = txy;
            *reinterpret_cast<float4 *>(syy + off[qd]) = tyy[qd];
        }
        __syncthreads();
        if (l == 0) hook();
        const float tau = stau[l];
#pragma unroll
        for (int qd = 0; qd < NQ; ++qd) {
            // u -= tau (Lxx' Txx + Lyy' Tyy + 2 Lxy' Txy)
            float X[6], Zu[6], Zd[6], Yu[4], Yc[4], Yd[4], U[4], f[6];
            quad_ext(txx[qd], X);
            quad_ext(*reinterpret_cast<const float4 *>(sxy + off[qd] - SW), Zu);
            quad_ext(*reinterpret_cast<const float4 *>(sxy + off[qd] + SW), Zd);
            f4_to(*reinterpret_cast<const float4 *>(syy + off[qd] - SW), Yu);
            f4_to(tyy[qd], Yc);
            f4_to(*reinterpret_cast<const float4 *>(syy + off[qd] + SW), Yd);
            f4_to(uo[qd], U);
#pragma unroll
            for (int j = 0; j < 6; ++j) f[j] = Zu[j] - Zd[j];  // column differences shared by neighbours
            float r[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float div = fmaf(0.5f, f[i] - f[i + 2],
                                       fmaf(-2.0f, X[i + 1], X[i] + X[i + 2]) + fmaf(-2.0f, Yc[i], Yu[i] + Yd[i]));
                r[i] = fmaf(-tau, div, U[i]);
                if (BOUNDARY && !((mask[qd] >> i) & 1u)) r[i] = U[i];
            }
            uo[qd] = make_float4(r[0], r[1], r[2], r[3]);
            *reinterpret_cast<float4 *>(su + off[qd]) = uo[qd];
        }
    }
}

}  // namespace fd4
