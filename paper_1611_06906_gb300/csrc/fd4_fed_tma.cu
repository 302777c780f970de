// FED cycle kernel with TMA staging (Sec. 3.4 Eq. 17, Sec. 3.5 Eq. 21):
// u <- u - tau_i L^T D L u, S = 2 or 4 explicit steps per launch on regions of
// 64 columns and RY = 64 or 32 rows, NQ = 1 or 2 row quads per thread, the quad
// arithmetic of fd4_quad.cuh.  S, RY and NQ form the schedule the autotuner
// times (fd4_autotune_batched); every schedule computes the same steps.
//
// Each tile's region of u and of the tensor field arrives by two tensor-map
// copies (cp.async.bulk.tensor) that one thread issues and an mbarrier counts
// in bytes: the hardware generates the addresses, zero-fills what lies outside
// the image, and the copies of the next two tiles overlap the current tile's
// steps.  The u box lands dense (64 rows of 256 B).  The tensor comes in one of
// two forms (the kernel's SOA parameter).  Inside the filter, the tensor build
// leaves the FED coefficient planes (mu3, q cos 2t, q sin 2t), whose box lands
// as three dense planes: 12 B per pixel, read by each thread as one float4 per
// plane and quad.  The float4 field (cos 2t, sin 2t, mu1, mu2) of fd4_fed_cycle
// lands as 64 rows of 16 quads of 64 B with the copy's 64-byte swizzle, which
// places the four pixels of quad q in the 16-byte slots i ^ ((q / 2) mod 4), so
// that the 16-byte reads of a quarter-warp hit distinct banks while each value
// goes straight to its pixel's register; the coefficients then follow per
// tile.  The issuing thread
// also records the tile's geometry in shared memory, so the other threads do
// no per-tile integer division.  Per-thread 16-byte copies
// (the cp.async kernels of fd4_fed.cu) reach about half of the HBM bandwidth on
// this staging; the bulk copies stream it.
#include <cuda.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "fd4_internal.h"
#include "fd4_quad.cuh"

namespace fd4 {

// Device status word of the FED kernels: FD4_ERR_TIMEOUT after a bounded wait
// on a tile's copies gave up.  Sticky until read with reset.
__device__ int g_fed_status;

namespace {

constexpr int TR = 64;                      // region width (columns); RY rows
constexpr int TSW = TR;                     // plane row stride (floats)
// Tiles in flight per block: the copies of the next two tiles run during the
// current tile's steps (one tile of 80 KB in flight per SM leaves the copies
// latency-bound at about half the HBM bandwidth).
constexpr int kAhead = 2;
template <int RY>
constexpr int t_quads() { return (TR / 4) * RY; }   // 16 quads x RY rows
template <int RY>
constexpr int t_plane() { return (RY + 2) * TSW; }  // one zero ring row above and below
template <int RY>
constexpr unsigned t_ubytes() { return TR * RY * 4; }   // u box
// tensor box: (cos 2t, sin 2t, mu1, mu2) per pixel, 16 B; or (SOA) the three
// FED coefficient planes (mu3, q cos 2t, q sin 2t), 12 B
template <int RY, bool SOA>
constexpr unsigned t_tbytes() { return SOA ? TR * RY * 12 : TR * RY * 16; }
// shared memory: tensor boxes x2 (1024-byte aligned) | u planes x3 | T_xy, T_yy
template <int RY, bool SOA>
constexpr size_t t_smem()
{
    return 1024 + kAhead * t_tbytes<RY, SOA>() + sizeof(float) * (kAhead + 1 + 2) * t_plane<RY>();
}
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded wait on a tile's copies

// 2-D maps of the two u planes {w, h}, the 3-D map of the tensor field
// {16, quads, h} and the 3-D map of the FED coefficient planes {w, h, 3}; their
// boxes have the region's rows.
struct TmaMaps {
    CUtensorMap u, tmp, ten, co;
};
// One image's maps for both region heights.
struct TmaMapSet {
    TmaMaps r64, r32;
};

// Bounded waits of one launch: the limit, and (self-test only) copies withheld
// so that the limit runs out.
struct FedWait {
    unsigned long long ns;
    int withhold;
};

__device__ __forceinline__ unsigned long long tma_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_mbar_init(uint64_t *m)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tma_expect(uint64_t *m, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool tma_try_wait(uint64_t *m, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of m, at most ns nanoseconds; false if it gave up.
__device__ __forceinline__ bool tma_wait(uint64_t *m, unsigned parity, unsigned long long ns)
{
    if (tma_try_wait(m, parity)) return true;
    const unsigned long long t0 = tma_now();
    while (!tma_try_wait(m, parity))
        if (tma_now() - t0 > ns) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *m)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(m))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *m)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(m))
        : "memory");
}
// Shared memory written or read through the generic proxy before the bulk copies overwrite it.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// A tensor map in global memory written by a kernel (generic proxy) before the copies read it.
__device__ __forceinline__ void fence_tensormap_acquire(const void *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// Tile shape of S steps on RY-row regions: (64 - 4S) x (RY - 4S) exact outputs.
template <int S, int RY>
constexpr int tma_shape() { return RY == 64 ? (S == 2 ? SHAPE_Q64_2 : SHAPE_Q64_4) : S; }

// Geometry of a staged tile, computed once by the thread that issues its copies.
struct TileGeo {
    int gx0, gy0;   // region origin in the image (gx0: a multiple of 4)
    int interior;   // the region lies inside the image
};

// Thread 0: the copies of the region of tile `local` of image d into u_dst (plane
// row 1) and the tensor box; the tile's geometry into *g.  withhold (self-test
// only): the barrier is armed for the bytes but no copy is issued.
template <int S, int RY, bool SOA>
__device__ __forceinline__ void tma_issue(const ImgDesc &d, int local, const TmaMaps &one, bool from_table,
                                          int parity, float *u_dst, void *t_dst, uint64_t *mbar, TileGeo *g,
                                          int withhold)
{
    constexpr int H = 2 * S, TOX = TR - 2 * H, TOY = RY - 2 * H;
    const int tiles_x = (d.w + TOX - 1) / TOX;
    const int ty = local / tiles_x;
    const int gx0 = (local - ty * tiles_x) * TOX - H, gy0 = ty * TOY - H;
    g->gx0 = gx0;
    g->gy0 = gy0;
    g->interior = gx0 >= 0 && gy0 >= 0 && gx0 + TR <= d.w && gy0 + RY <= d.h;
    const TmaMaps *m = &one;
    if (from_table) {
        const TmaMapSet *set = reinterpret_cast<const TmaMapSet *>(d.maps);
        m = RY == 64 ? &set->r64 : &set->r32;
    }
    const CUtensorMap *mu = parity ? &m->tmp : &m->u;
    const CUtensorMap *mt = SOA ? &m->co : &m->ten;
    if (from_table) {
        fence_tensormap_acquire(mu);
        fence_tensormap_acquire(mt);
    }
    fence_async_smem();
    tma_expect(mbar, t_ubytes<RY>() + t_tbytes<RY, SOA>());
    if (withhold) return;
    tma_load_2d(u_dst + TSW, mu, gx0, gy0, mbar);  // x: 4 gx0 bytes, a multiple of 16
    if (SOA)
        tma_load_3d(t_dst, mt, gx0, gy0, 0, mbar);  // x: 4 gx0 bytes, as above
    else
        tma_load_3d(t_dst, mt, 0, gx0 >> 2, gy0, mbar);  // x: 0; the quad index may be -1
}

// NQ quads per thread: 16 RY / NQ threads, thread (row ry, quad column q) owns
// the quads of rows ry + i RY / NQ, i < NQ.  With NQ = 2 a block barrier spans
// half the warps and each thread has two independent quads in flight.  A block
// of 64-row regions takes one SM (217 KB of shared memory); two blocks of
// 32-row regions share one.
template <int S, int NQ, int RY, bool SOA>
__global__ void __launch_bounds__(t_quads<RY>() / NQ, RY == 64 ? 1 : 2)
    k_fed_tma(Imgs I, StepTaus taus, int parity, const __grid_constant__ TmaMaps one, FedWait wt)
{
    constexpr int H = 2 * S, TOX = TR - 2 * H, TOY = RY - 2 * H, SHAPE = tma_shape<S, RY>(), NU = kAhead + 1;
    constexpr int NT = t_quads<RY>() / NQ, TPLANE = t_plane<RY>();
    constexpr unsigned TBYTES = t_tbytes<RY, SOA>();
    static_assert(TOX % 4 == 0 && H % 4 == 0 && TOY > 0, "whole quads in the exact interior");
    extern __shared__ unsigned char tma_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)tma_raw + 1023) & ~(uintptr_t)1023);
    // tensor boxes: tile j of this block in box j % kAhead (RY rows x 64 pixels x 16 B,
    // or SOA: 3 planes x RY rows x 64 pixels x 4 B)
    float *planes = reinterpret_cast<float *>(base + kAhead * TBYTES);  // u planes x NU | T_xy | T_yy
    float *sxy = planes + NU * TPLANE, *syy = planes + (NU + 1) * TPLANE;
    __shared__ uint64_t mbar[kAhead];     // tile j waits on mbar[j % kAhead]
    __shared__ float stau[8];
    __shared__ ImgDesc sd[NU];            // tile j's descriptor in sd[j % NU]
    __shared__ int s_local[NU];
    __shared__ TileGeo sgeo[NU];
    __shared__ int abort_flag;
    __shared__ TileCache tcache;
    const int tid = threadIdx.x;
    const bool from_table = I.table != nullptr;
    for (int i = tid; i < (NU + 2) * TPLANE; i += NT) planes[i] = 0.0f;  // the ring rows stay zero
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) stau[i] = taus.t[i];
        abort_flag = 0;
        tc_reset(tcache);
        for (int i = 0; i < kAhead; ++i) tma_mbar_init(&mbar[i]);
    }
    const int q = tid & 15, ry0 = tid >> 4, tswz = (q >> 1) & 3;
    int off[NQ], rowq[NQ];
    bool writes[NQ];
#pragma unroll
    for (int qd = 0; qd < NQ; ++qd) {
        rowq[qd] = ry0 + qd * (RY / NQ);
        off[qd] = (rowq[qd] + 1) * TSW + 4 * q;  // this quad in a plane
        // the quad lies in the exact interior of every tile: rows H .. H + TOY - 1, columns H .. H + TOX - 1
        writes[qd] = rowq[qd] >= H && rowq[qd] < H + TOY && 4 * q >= H && 4 * q < H + TOX;
    }
    const int ntiles = I.tiles, G = gridDim.x;
    __syncthreads();
    // prologue: the copies of the block's first kAhead tiles
    if (tid == 0)
        for (int j = 0; j < kAhead; ++j) {
            const int tj = blockIdx.x + j * G;
            if (tj >= ntiles) break;
            find_tile_cached(I, SHAPE, tj, tcache, sd[j], s_local[j]);
            tma_issue<S, RY, SOA>(sd[j], s_local[j], one, from_table, parity, planes + j * TPLANE,
                                  base + j * TBYTES, &mbar[j], &sgeo[j], wt.withhold);
        }
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, ++j) {
        const int bj = j % kAhead, uj = j % NU;
        if (!tma_wait(&mbar[bj], (unsigned)(j / kAhead) & 1u, wt.ns)) abort_flag = 1;
        __syncthreads();  // tile j has landed; every warp is past tile j - 1
        if (abort_flag) break;
        const ImgDesc &d = sd[uj];
        const int w = d.w, h = d.h;
        const int gx = sgeo[uj].gx0 + 4 * q;
        const bool interior = sgeo[uj].interior != 0;
        float *su = planes + uj * TPLANE;
        float4 uq[NQ];
        unsigned mask[NQ];
        QuadCoef k[NQ];
#pragma unroll
        for (int qd = 0; qd < NQ; ++qd) {
            const int gy = sgeo[uj].gy0 + rowq[qd];
            uq[qd] = *reinterpret_cast<const float4 *>(su + off[qd]);
            mask[qd] = 0u;
            if (!interior) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int x = gx + i;
                    mask[qd] |= (x >= 0 && x < w && gy >= 0 && gy < h ? 1u : 0u) << i;
                    mask[qd] |= (x >= 1 && x <= w - 2 ? 1u : 0u) << (4 + i);
                }
                mask[qd] |= (gy >= 1 && gy <= h - 2 ? 1u : 0u) << 8;
            }
            if (SOA) {
                // the three coefficient planes of the box, dense rows of 64
                // floats: a quarter-warp reads 128 contiguous bytes of each
                const float *tb = reinterpret_cast<const float *>(base + bj * TBYTES) + rowq[qd] * TR + 4 * q;
                const float4 qs4 = *reinterpret_cast<const float4 *>(tb + 2 * RY * TR);
                k[qd].m = *reinterpret_cast<const float4 *>(tb);
                k[qd].qc = *reinterpret_cast<const float4 *>(tb + RY * TR);
                k[qd].qs = qs4;
                k[qd].qs2 = make_float4(qs4.x + qs4.x, qs4.y + qs4.y, qs4.z + qs4.z, qs4.w + qs4.w);
                continue;
            }
            // The copy's 64-byte swizzle put pixel i of quad q in 16-byte slot
            // i ^ r of the quad, r = (q / 2) mod 4: the 8 lanes of a quarter-warp
            // then read 8 distinct 16-byte bank groups, and every value lands in
            // its pixel's register.
            const float4 *tq =
                reinterpret_cast<const float4 *>(base + bj * TBYTES + (size_t)rowq[qd] * (TR * 16)) + 4 * q;
            float4 v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = tq[i ^ tswz];
            float mm[4], qc[4], qs[4], q2[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 tt = v[i];  // (cos 2t, sin 2t, mu1, mu2)
                const float qq = 0.25f * (tt.z - tt.w);
                mm[i] = 0.5f * (tt.z + tt.w);
                qc[i] = qq * tt.x;
                qs[i] = qq * tt.y;
                q2[i] = qs[i] + qs[i];
            }
            k[qd].m = make_float4(mm[0], mm[1], mm[2], mm[3]);
            k[qd].qc = make_float4(qc[0], qc[1], qc[2], qc[3]);
            k[qd].qs = make_float4(qs[0], qs[1], qs[2], qs[3]);
            k[qd].qs2 = make_float4(q2[0], q2[1], q2[2], q2[3]);
        }
        // Tile j + kAhead goes into box bj and plane (j + kAhead) % NU, once every
        // thread has read box bj (above) and is past tile j - 1, the last user of
        // that plane and of its descriptor slot: after the first step's T barrier.
        const int ta = t + kAhead * G;
        const auto issue = [&]() {
            if (tid == 0 && ta < ntiles) {
                const int ua = (j + kAhead) % NU;
                find_tile_cached(I, SHAPE, ta, tcache, sd[ua], s_local[ua]);
                tma_issue<S, RY, SOA>(sd[ua], s_local[ua], one, from_table, parity, planes + ua * TPLANE,
                                      base + bj * TBYTES, &mbar[bj], &sgeo[ua], wt.withhold);
            }
        };
        if (taus.n < 1) {
            __syncthreads();
            issue();
        }
        if (interior) quad_steps_n<false, TSW, NQ>(su, sxy, syy, stau, taus.n, off, k, mask, uq, issue);
        else quad_steps_n<true, TSW, NQ>(su, sxy, syy, stau, taus.n, off, k, mask, uq, issue);
        // the exact interior: rows H .. H + TOY - 1, columns H .. H + TOX - 1 (whole quads)
#pragma unroll
        for (int qd = 0; qd < NQ; ++qd) {
            const int gy = sgeo[uj].gy0 + rowq[qd];
            if (writes[qd] && gy < h) {
                float *dst = (parity ? d.u : d.tmp) + (size_t)gy * d.pitch + gx;
                const float4 un = uq[qd];
                if (gx + 3 < w) {
                    *reinterpret_cast<float4 *>(dst) = un;
                } else {
                    if (gx < w) dst[0] = un.x;
                    if (gx + 1 < w) dst[1] = un.y;
                    if (gx + 2 < w) dst[2] = un.z;
                }
            }
        }
    }
    if (abort_flag && tid == 0) {
        atomicExch(&g_fed_status, FD4_ERR_TIMEOUT);
        // the copies still in flight (tiles j .. j + kAhead - 1), each wait again bounded
        for (int i = 0; i < kAhead; ++i) {
            const int jj = j + i;
            if (blockIdx.x + jj * G < ntiles) tma_wait(&mbar[jj % kAhead], (unsigned)(jj / kAhead) & 1u, wt.ns);
        }
    }
}

// Map table writer: a chunk of per-image tensor map sets passed as kernel parameters.
constexpr int kMapChunk = 16;
struct MapChunk {
    int first, n;
    TmaMapSet m[kMapChunk];
};
__global__ void k_put_maps(const __grid_constant__ MapChunk c, TmaMapSet *table)
{
    const int i = blockIdx.x, j = threadIdx.x;  // set i of the chunk, its 16-byte word j
    if (i < c.n && j < (int)(sizeof(TmaMapSet) / 16)) {
        reinterpret_cast<uint4 *>(&table[c.first + i])[j] = reinterpret_cast<const uint4 *>(&c.m[i])[j];
        asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
    }
}

// The four maps of one image for regions of `rows` rows (zero fill outside the image).
int make_maps(const ImgDesc &d, int rows, TmaMaps *m)
{
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return 1;
    const cuuint64_t dim2[2] = {(cuuint64_t)d.w, (cuuint64_t)d.h};
    const cuuint64_t str2[1] = {(cuuint64_t)d.pitch * 4};
    const cuuint32_t box2[2] = {TR, (cuuint32_t)rows};
    const cuuint32_t one2[2] = {1, 1};
    if (enc(&m->u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)d.u, dim2, str2, box2, one2,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    if (enc(&m->tmp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)d.tmp, dim2, str2, box2, one2,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    // tensor: floats of one quad (64 bytes) x quads of a row x rows, so that the
    // 64-byte swizzle permutes the four pixels of each quad; the pitch is a
    // multiple of 4, so the last (partial) quad of a row lies within the pitch
    const cuuint64_t dimt[3] = {16, (cuuint64_t)(d.w + 3) / 4, (cuuint64_t)d.h};
    const cuuint64_t strt[2] = {64, (cuuint64_t)d.pitch * 16};
    const cuuint32_t boxt[3] = {16, TR / 4, (cuuint32_t)rows};
    const cuuint32_t one3[3] = {1, 1, 1};
    if (enc(&m->ten, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)d.tensor, dimt, strt, boxt, one3,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    // FED coefficient planes: columns x rows x the three planes (they lie in the
    // 16 B per pixel of the tensor plane)
    const cuuint64_t dimc[3] = {(cuuint64_t)d.w, (cuuint64_t)d.h, 3};
    const cuuint64_t strc[2] = {(cuuint64_t)d.pitch * 4, (cuuint64_t)fed_coef_plane(d.h, d.pitch) * 4};
    const cuuint32_t boxc[3] = {TR, (cuuint32_t)rows, 3};
    if (enc(&m->co, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)d.tensor, dimc, strc, boxc, one3,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    return 0;
}

int make_map_set(const ImgDesc &d, TmaMapSet *m) { return make_maps(d, 64, &m->r64) || make_maps(d, 32, &m->r32); }

template <int S, int NQ, int RY, bool SOA>
int set_tma_smem()
{
    static int attr_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (attr_dev != dev) {
        if (cudaFuncSetAttribute(k_fed_tma<S, NQ, RY, SOA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)t_smem<RY, SOA>()) != cudaSuccess)
            return 1;
        attr_dev = dev;
    }
    return 0;
}

template <int S, int NQ, int RY, bool SOA>
int launch_tma_k(const Imgs &I, const StepTaus &t, int parity, const TmaMaps &one, const FedWait &wt,
                 cudaStream_t st)
{
    if (set_tma_smem<S, NQ, RY, SOA>()) return 1;
    constexpr int NT = t_quads<RY>() / NQ;
    constexpr size_t smem = t_smem<RY, SOA>();
    const int grid = persistent_grid((const void *)k_fed_tma<S, NQ, RY, SOA>, NT, smem, I.tiles);
    k_fed_tma<S, NQ, RY, SOA><<<grid, NT, smem, st>>>(I, t, parity, one, wt);
    return cudaGetLastError() != cudaSuccess;
}

template <int S, int RY, bool SOA>
int launch_tma_q(const Imgs &I, const StepTaus &t, int parity, const TmaMaps &one, const FedWait &wt, int quads,
                 cudaStream_t st)
{
    return quads == 1 ? launch_tma_k<S, 1, RY, SOA>(I, t, parity, one, wt, st)
                      : launch_tma_k<S, 2, RY, SOA>(I, t, parity, one, wt, st);
}

template <int S>
int launch_tma_sched(const HostBatch &B, const double *tau, int k, int parity, const FedSched &sch, const FedWait &wt,
                     cudaStream_t st)
{
    StepTaus t{};
    t.n = k;
    for (int i = 0; i < k; ++i) t.t[i] = (float)tau[i];
    Imgs I = B.I;
    const bool r32 = sch.rows == 32;
    I.tiles = B.tiles[r32 ? tma_shape<S, 32>() : tma_shape<S, 64>()];
    TmaMapSet set;
    memset(&set, 0, sizeof(set));
    if (!I.table && make_map_set(I.one, &set)) return 1;
    const TmaMaps &one = r32 ? set.r32 : set.r64;
    if (B.fed_soa)
        return r32 ? launch_tma_q<S, 32, true>(I, t, parity, one, wt, sch.quads, st)
                   : launch_tma_q<S, 64, true>(I, t, parity, one, wt, sch.quads, st);
    return r32 ? launch_tma_q<S, 32, false>(I, t, parity, one, wt, sch.quads, st)
               : launch_tma_q<S, 64, false>(I, t, parity, one, wt, sch.quads, st);
}

}  // namespace

EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

size_t tma_maps_bytes() { return sizeof(TmaMapSet); }

template <bool SOA>
int prepare_tma_kernels_of()
{
    return set_tma_smem<2, 1, 64, SOA>() || set_tma_smem<4, 1, 64, SOA>() || set_tma_smem<2, 2, 64, SOA>() ||
           set_tma_smem<4, 2, 64, SOA>() || set_tma_smem<2, 1, 32, SOA>() || set_tma_smem<4, 1, 32, SOA>() ||
           set_tma_smem<2, 2, 32, SOA>() || set_tma_smem<4, 2, 32, SOA>();
}

int prepare_tma_kernels() { return prepare_tma_kernels_of<false>() || prepare_tma_kernels_of<true>(); }

// Writes the map sets of the n descriptors (their maps fields point into a
// device table) with kernels on st.
int launch_put_maps(const ImgDesc *h_descs, int n, void *d_table, cudaStream_t st)
{
    thread_local static MapChunk c;  // 16 KB: kept off the stack
    for (int first = 0; first < n; first += kMapChunk) {
        c.first = first;
        c.n = n - first < kMapChunk ? n - first : kMapChunk;
        for (int i = 0; i < c.n; ++i)
            if (make_map_set(h_descs[first + i], &c.m[i])) return 1;
        k_put_maps<<<c.n, (int)(sizeof(TmaMapSet) / 16), 0, st>>>(c, (TmaMapSet *)d_table);
    }
    return cudaGetLastError() != cudaSuccess;
}

// One launch of k steps (k <= S) of the TMA kernel over the batch.  Batches
// (I.table) take each image's maps from its descriptor; a single inline image
// gets its maps as a kernel parameter.
template <int S>
int launch_fed_tma(const HostBatch &B, const double *tau, int k, int parity, const FedSched &sch, cudaStream_t st)
{
    return launch_tma_sched<S>(B, tau, k, parity, sch, FedWait{kWaitNs, 0}, st);
}

template int launch_fed_tma<2>(const HostBatch &, const double *, int, int, const FedSched &, cudaStream_t);
template int launch_fed_tma<4>(const HostBatch &, const double *, int, int, const FedSched &, cudaStream_t);

}  // namespace fd4

extern "C" int fd4_device_status(int *status, int reset)
{
    if (!status) return FD4_ERR_BAD_ARG;
    if (cudaMemcpyFromSymbol(status, fd4::g_fed_status, sizeof(int)) != cudaSuccess) return FD4_ERR_CUDA;
    if (reset) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(fd4::g_fed_status, &zero, sizeof(int)) != cudaSuccess) return FD4_ERR_CUDA;
    }
    return FD4_OK;
}

extern "C" int fd4_selftest_fed_wait_timeout(float *d_u, int w, int h, int pitch, const float *d_tensor,
                                             void *d_ws, size_t ws_bytes, int *status, fd4_stream_t stream)
{
    using namespace fd4;
    int rc;
    if (!status || !d_tensor) return FD4_ERR_BAD_ARG;
    if ((rc = check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if ((uintptr_t)d_tensor & 15u) return FD4_ERR_ALIGN;
    if (!d_ws || ((uintptr_t)d_ws & 255u)) return d_ws ? FD4_ERR_ALIGN : FD4_ERR_BAD_ARG;
    if (ws_bytes < ws_fed_bytes(h, pitch)) return FD4_ERR_WS_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    const int zero = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpyToSymbol(g_fed_status, &zero, sizeof(int)) != cudaSuccess)
        return FD4_ERR_CUDA;
    ImgDesc d{};
    d.u = d_u;
    d.tmp = (float *)((char *)d_ws + kHeaderBytes);
    d.tensor = (float4 *)d_tensor;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    const double tau[2] = {0.01, 0.01};
    // every wait of the launch gives up after 10 ms: the copies are withheld,
    // so the tile's barrier never completes; nothing is ever in flight
    if (launch_tma_sched<2>(single_batch(d), tau, 2, 0, kDefaultSched, FedWait{10000000ull, 1}, st) ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FD4_ERR_CUDA;
    return fd4_device_status(status, 1);
}
