// Learned scale selector (no counterpart in the paper: the paper selects the
// scale with the vesselness argmax of Sec. 3.3; this network predicts that
// argmax and the plain sweep checks it).
//
// Network: four dilated 3 x 3 convolutions (dilations 1, 2, 4, 8; channels
// 1 -> 32 -> 32 -> 32 -> 16), ReLU between them, softmax over the first n_bins
// (<= 16) outputs, one bin per scale of the set (8 or 12 in the workloads).
// Activations are NHWC bf16 (16 channels for the input layer, 32 after);
// weights bf16; accumulation FP32 in tensor memory.
//
// Convolution as implicit GEMM on the 5th-generation tensor cores: a tile is
// 128 consecutive output pixels of one image row (the MMA's M = 128); the
// three input rows y - d, y, y + d (with a d-pixel margin) sit in shared
// memory as 16-byte channel chunks laid out pixel-contiguous, so the A operand
// of tap (ky, kx) is a row buffer shifted by kx * d pixels -- a plain K-major
// no-swizzle descriptor, no im2col copy.  A block walks down one residue class
// of the rows modulo d, so consecutive tiles share two input rows and each
// tile copies one new row (cp.async, during the previous tile's MMAs).  B (the
// weights of all nine taps) is staged once per block.  One thread issues
// 9 * CI/16 MMAs of 128 x CO x 16, commits them to an mbarrier, and the four
// warps read the FP32 accumulator back from their TMEM lanes for the epilogue
// (bias + ReLU + bf16, or at inference the argmax bin and its probability).
// The weight gradient is a tensor-core product too, with the pixels as the
// reduction dimension (k_sel_wgrad_tc).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "fd4_internal.h"
#include "fd4_tc.cuh"

namespace fd4 {
namespace {

constexpr int TM = 128;           // output pixels per tile (MMA M)
constexpr int CT = 128;           // threads: warp w owns TMEM lanes 32w .. 32w+31
constexpr int kMaxDil = 8;

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

enum ConvMode { CONV_RELU_BF16 = 0, CONV_LOGITS_F32 = 1, CONV_MASK_BF16 = 2, CONV_PREDICT = 3 };

// Activations (bf16) are stored row-planar with their own pitch `apitch` (a
// multiple of 8 pixels, pixels w .. apitch - 1 zero): row y of image i holds
// C / 8 chunk planes of apitch pixels x 8 channels (16 bytes), so that
// channels 8j .. 8j + 7 of pixel x are at
// ((i * h + y) * apitch * C / 8 + j * apitch + x) * 8.  A row's run of pixels
// in one plane is contiguous: one tensor-map copy moves a window of an input
// row in all its planes, and a warp's 16-byte stores of one plane are
// contiguous.
__host__ __device__ inline size_t act_off(long long aimg_stride, int img, int y, int apitch, int cj, int j, int x)
{
    return (((size_t)img * (size_t)aimg_stride + (size_t)y * apitch) * cj + (size_t)j * apitch + x) * 8;
}
__host__ __device__ inline int act_pitch(int w) { return (w + 7) / 8 * 8; }

struct ConvArgs {
    const __nv_bfloat16 *in;    // row-planar, CI channels (input of layer 0: one stored plane, the rest zero)
    void *out;                  // row-planar CO channels (bf16), or n_out floats per pixel (fp32 logits)
    const uint4 *wts;           // weights in tile layout: [tap][ci / 8][co] x 16 bytes
    const float *bias;          // CO floats, nullable
    const __nv_bfloat16 *mask;  // CONV_MASK_BF16: row-planar, CO channels; output zeroed where mask <= 0
    uint8_t *idx;               // CONV_PREDICT: argmax of the first n_out outputs per pixel
    float *conf;                // CONV_PREDICT: its softmax probability (nullable)
    int n_img, w, h, d;
    int pitch;                  // logits / idx / conf: elements per row
    int apitch;                 // activations: pixels per row (act_pitch(w))
    long long img_stride;       // h * pitch
    long long aimg_stride;      // h * apitch
    int n_out;                  // CONV_LOGITS_F32 / CONV_PREDICT: outputs used per pixel
    int in_cj;                  // chunk planes stored per input row (<= CI / 8; the missing ones read as zero)
    int seg_rows;               // output rows of one residue class per work unit
    int *status;                // FD4_ERR_TIMEOUT if a wait gives up
    int withhold_commit;        // self-test only: issue no MMA, so the waits run out
};

// Warps of a convolution block: the epilogue warps (a TMEM lane quarter and a
// group of 16 output channels each: 8 for 32 outputs, 4 for 16), then the
// copy warp and the MMA warps: one for 32 outputs (the epilogue is the longer
// stage), two for 16 (even and odd input rows; issuing is the longer stage).
__host__ __device__ constexpr int conv_epi_warps(int CO) { return CO == 32 ? 8 : 4; }
__host__ __device__ constexpr int conv_mma_warps(int CO) { return CO == 32 ? 1 : 2; }
__host__ __device__ constexpr int conv_threads(int CO) { return (conv_epi_warps(CO) + 1 + conv_mma_warps(CO)) * 32; }
constexpr int kSlots = 5;          // input rows staged per block
constexpr uint64_t kConvWaitNs = 1000000000ull;  // bounded waits: one second
// A staged row holds pixels x0 - 8 .. x0 + 135 of each plane: 18 segments of
// 8 pixels (128 bytes), one tensor-map copy.  Tap kx of dilation d reads
// pixels from x0 + (kx - 1) d, at offset 8 + (kx - 1) d.
constexpr int kSegPx = 8;
constexpr int kWinPx = 144;
static_assert(TM + 2 * kMaxDil <= kWinPx && kMaxDil <= kSegPx, "the window covers the tile and its margins");

__host__ __device__ constexpr uint32_t conv_slot_bytes(int cj) { return (uint32_t)cj * kWinPx * 16u; }
// weights | row ring (plus 128 bytes to align the base)
__host__ __device__ constexpr size_t conv_smem_bytes(int CI, int CO)
{
    return 128 + (size_t)16 * 9 * (CI / 8) * CO + (size_t)kSlots * conv_slot_bytes(CI / 8);
}
// TMEM columns: two accumulators of 3 CO columns, rounded up to a power of two
__host__ __device__ constexpr uint32_t conv_tmem_cols(int CO) { return 6 * CO <= 128 ? 128u : 256u; }

// Work units of a convolution: (image, 128-pixel column tile, residue class of
// the rows modulo the dilation d, segment of seg rows of that class).
__host__ __device__ inline long long conv_units(int n_img, int w, int h, int d, int seg)
{
    const int tiles_x = (w + TM - 1) / TM;
    const int cls = (h + d - 1) / d;  // rows of the longest residue class
    const int segs = (cls + seg - 1) / seg;
    return (long long)n_img * tiles_x * d * segs;
}

struct ConvUnit {
    int img, x0, rho, k0, k1;  // output class positions k0 .. k1 - 1, rows y = rho + k d
};
__device__ __forceinline__ bool conv_unit(const ConvArgs &a, long long u, int segs, int tiles_x, ConvUnit &c)
{
    const int seg = (int)(u % segs);
    long long rest = u / segs;
    c.rho = (int)(rest % a.d);
    rest /= a.d;
    c.x0 = (int)(rest % tiles_x) * TM;
    c.img = (int)(rest / tiles_x);
    c.k0 = seg * a.seg_rows;
    const int kmax = c.rho < a.h ? (a.h - 1 - c.rho) / a.d + 1 : 0;
    c.k1 = min(c.k0 + a.seg_rows, kmax);
    return c.k0 < c.k1;
}

template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[N])
{
    if constexpr (N == 32) {
        tc::tmem_ld_x32(taddr, v);
    } else {
        tc::tmem_ld_x16(taddr, v);
    }
}

// Implicit-GEMM 3 x 3 dilated convolution on the tensor cores, one input row
// at a time, with warp roles.  A block walks units (one residue class of the
// rows modulo d, a 128-pixel column tile, a segment of its rows); output rows
// k0 .. k1 - 1 of a unit read input rows k0 - 1 .. k1 (class positions).  For
// input row r the MMA warp computes, in one TMEM accumulator of 3 CO columns,
//   D_r[p][ky CO + co] = sum_kx sum_ci X_r[p + (kx - 1) d][ci] W[ky][kx][co][ci]
// as 3 kx x CI / 16 MMAs of 128 x 3 CO x 16: A is the staged row at a
// (kx - 1) d pixel shift (a K-major no-swizzle operand: LBO = one chunk plane,
// SBO = 8 pixels), B the weights of the three ky taps stacked along N.
// Output row k is D_{k-1}[ky = 0] + D_k[ky = 1] + D_{k+1}[ky = 2]: the four
// epilogue warps (a pixel per thread, its TMEM lane) carry the two partial
// sums of the rows still open in registers.  The copy warp streams input rows
// into a ring of kSlots buffers (one tensor-map copy per row, zero fill
// outside the image); the MMA warp issues a row's MMAs as soon as its copy
// and a free accumulator are there, into the accumulator the epilogue is not
// reading (with two MMA warps, one per accumulator, alternate rows).  Handoffs are mbarriers: full (copy landed), empty (MMAs of the
// slot done), acc_full (accumulator written), acc_empty (epilogue has read
// it).  Every wait is bounded (one second): on timeout the kernel records
// FD4_ERR_TIMEOUT, the roles stop, the copies and MMAs in flight are waited
// for (bounded), the TMEM is freed and the kernel returns.
template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(conv_threads(CO), 2) k_conv_tc(const __grid_constant__ CUtensorMap xmap, ConvArgs a)
{
    constexpr int CJ = CI / 8;  // 16-byte channel chunks per pixel
    constexpr int NN = 3 * CO;  // MMA N: the three ky taps
    constexpr int NEPI = conv_epi_warps(CO);
    constexpr int kThreads = conv_threads(CO);
    constexpr uint32_t kCols = conv_tmem_cols(CO);
    constexpr uint32_t slot_bytes = conv_slot_bytes(CJ);
    extern __shared__ unsigned char conv_raw[];
    __shared__ __align__(8) uint64_t full_bar[kSlots];
    __shared__ __align__(8) uint64_t empty_bar[kSlots];
    __shared__ __align__(8) uint64_t accf_bar[2];
    __shared__ __align__(8) uint64_t acce_bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ float bias_s[CO];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)conv_raw + 127) & ~(uintptr_t)127);
    uint4 *Bs = reinterpret_cast<uint4 *>(base);        // [kx][ci / 8][ky][co] x 16 bytes
    unsigned char *ring = base + 16 * 9 * CJ * CO;      // kSlots x CJ planes x kWinPx pixels x 16 bytes
    const int d = a.d;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights [tap][ci / 8][co] -> [kx][ci / 8][ky][co]: the ky taps of one
    // (kx, chunk) are N-contiguous
    for (int i = tid; i < 9 * CJ * CO; i += kThreads) {
        const int co = i % CO, j = (i / CO) % CJ, tap = i / (CO * CJ);
        const int ky = tap / 3, kx = tap - 3 * (tap / 3);
        Bs[((kx * CJ + j) * 3 + ky) * CO + co] = a.wts[i];
    }
    // planes the input does not store are zero in every slot (no copy writes them)
    for (int s = 0; s < kSlots; ++s)
        for (int i = a.in_cj * kWinPx + tid; i < CJ * kWinPx; i += kThreads)
            reinterpret_cast<uint4 *>(ring + s * slot_bytes)[i] = make_uint4(0u, 0u, 0u, 0u);
    // (the prediction masks the bins from n_out on with a bias of -inf)
    for (int c = tid; c < CO; c += kThreads)
        bias_s[c] = (MODE == CONV_PREDICT && c >= a.n_out) ? -INFINITY : (a.bias ? a.bias[c] : 0.0f);
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, kCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) {
            tc::mbar_init(&full_bar[s], 1);
            tc::mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&accf_bar[b], 1);
            tc::mbar_init(&acce_bar[b], NEPI);  // one arrival per epilogue warp
        }
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    tc::fence_proxy_async();  // the weights and zero planes, written by this proxy, are read by the MMAs
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const int tiles_x = (a.w + TM - 1) / TM;
    const int cls = (a.h + d - 1) / d;
    const int segs = (cls + a.seg_rows - 1) / a.seg_rows;
    const long long total = conv_units(a.n_img, a.w, a.h, d, a.seg_rows);
    const uint32_t ring_s = tc::smem_u32(ring);

    if (warp == NEPI) {
        // ---- copy warp: input rows into the ring
        if (lane == 0) {
            uint32_t q = 0;  // rows of this block so far: slot q % kSlots, use q / kSlots
            bool stop = false;
            for (long long u = blockIdx.x; u < total && !stop; u += gridDim.x) {
                ConvUnit c;
                if (!conv_unit(a, u, segs, tiles_x, c)) continue;
                for (int r = c.k0 - 1; r <= c.k1; ++r, ++q) {
                    const uint32_t s = q % kSlots, n = q / kSlots;
                    if (abort_flag || (n > 0 && !tc::mbar_wait_bounded(&empty_bar[s], (n - 1) & 1u, kConvWaitNs))) {
                        abort_flag = 1;
                        stop = true;
                        break;
                    }
                    tc::mbar_expect_tx(&full_bar[s], (uint32_t)a.in_cj * kWinPx * 16u);
                    tc::tma_load_5d(ring_s + s * slot_bytes, &xmap, 0, c.x0 / kSegPx - 1, 0, c.rho + r * d, c.img,
                                    &full_bar[s]);
                }
            }
            // every copy issued has landed before the block ends
            for (uint32_t s = 0; s < kSlots && s < q; ++s)
                tc::mbar_wait_bounded(&full_bar[s], ((q - 1 - s) / kSlots) & 1u, kConvWaitNs);
        }
    } else if (warp > NEPI) {
        // ---- MMA warps: with two, the first takes the even rows (accumulator
        // 0), the second the odd rows (accumulator 1); a row's MMAs are issued
        // by one thread, in order
        constexpr int NMMA = conv_mma_warps(CO);
        const uint32_t mine = (uint32_t)(warp - NEPI - 1);
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(TM, NN);
            const uint64_t adesc0 = tc::sdesc_kmajor(ring_s, (uint32_t)(kWinPx * 16), 128);
            const uint64_t bdesc0 = tc::sdesc_kmajor(tc::smem_u32(Bs), (uint32_t)(NN * 16), 128);
            uint32_t q = 0, committed = 0;
            bool stop = false;
            for (long long u = blockIdx.x; u < total && !stop; u += gridDim.x) {
                ConvUnit c;
                if (!conv_unit(a, u, segs, tiles_x, c)) continue;
                for (int r = c.k0 - 1; r <= c.k1; ++r, ++q) {
                    const uint32_t s = q % kSlots, n = q / kSlots, b = q & 1u, nb = q >> 1;
                    if (NMMA == 2 && b != mine) continue;
                    if (abort_flag || !tc::mbar_wait_bounded(&full_bar[s], n & 1u, kConvWaitNs) ||
                        (nb > 0 && !tc::mbar_wait_bounded(&acce_bar[b], (nb - 1) & 1u, kConvWaitNs))) {
                        abort_flag = 1;
                        stop = true;
                        break;
                    }
                    if (a.withhold_commit) continue;
                    tc::fence_after_sync();
                    const uint32_t srow = s * (slot_bytes >> 4) + (uint32_t)(kSegPx - d);
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                        for (int kk = 0; kk < CI / 16; ++kk) {
                            // descriptor start addresses advance in 16-byte units
                            const uint64_t ad = adesc0 + (uint64_t)(srow + (uint32_t)(2 * kk * kWinPx + kx * d));
                            const uint64_t bd = bdesc0 + (uint64_t)((kx * CJ + 2 * kk) * NN);
                            tc::mma_bf16(tmem + b * NN, ad, bd, idesc, (kx | kk) != 0 ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(&empty_bar[s]);
                    tc::mma_commit(&accf_bar[b]);
                    ++committed;
                }
            }
            // the MMAs issued are complete before the TMEM is freed: the last
            // commit on each accumulator this warp feeds
            if (NMMA == 2) {
                if (committed > 0) tc::mbar_wait_bounded(&accf_bar[mine], (committed - 1) & 1u, kConvWaitNs);
            } else {
                for (uint32_t b = 0; b < 2 && b < committed; ++b)
                    tc::mbar_wait_bounded(&accf_bar[b], ((committed - 1 - b) / 2) & 1u, kConvWaitNs);
            }
        }
    } else {
        // ---- epilogue warps: lane quarter warp % 4 of the accumulators,
        // output channels 16 g .. 16 g + 15 with g = warp / 4 (the running sums
        // stay in registers)
        const int lq = warp & 3, g = warp >> 2;
        const int i = lq * 32 + lane;  // tile pixel = TMEM lane
        uint32_t q = 0;
        bool stop = false;
        for (long long u = blockIdx.x; u < total && !stop; u += gridDim.x) {
            ConvUnit c;
            if (!conv_unit(a, u, segs, tiles_x, c)) continue;
            float accA[16], accB[16];  // partial sums of output rows r - 1 and r
#pragma unroll
            for (int k = 0; k < 16; ++k) accA[k] = accB[k] = 0.0f;
            const int gx = c.x0 + i;
            for (int r = c.k0 - 1; r <= c.k1; ++r, ++q) {
                const uint32_t b = q & 1u, nb = q >> 1;
                if (abort_flag || !tc::mbar_wait_bounded(&accf_bar[b], nb & 1u, kConvWaitNs)) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + b * NN;
                const bool emit = r - 1 >= c.k0;
                const int y = c.rho + (r - 1) * d;
                {
                    // ky = 2 closes output row r - 1, ky = 1 adds to row r, ky = 0 opens row r + 1
                    uint32_t r2[16], r1[16], r0[16];
                    tc::tmem_ld_x16_async(taddr + 2 * CO + 16 * g, r2);
                    tc::tmem_ld_x16_async(taddr + CO + 16 * g, r1);
                    tc::tmem_ld_x16_async(taddr + 16 * g, r0);
                    tc::tmem_wait_ld();
                    // the accumulator is read: release it to the MMA warp
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&acce_bar[b]))
                                     : "memory");
                    float v[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        v[k] = __uint_as_float(r2[k]) + accA[k];
                        accA[k] = accB[k] + __uint_as_float(r1[k]);
                        accB[k] = __uint_as_float(r0[k]);
                    }
                    if (!emit) continue;
                    // this pixel's 16 bytes in chunk plane j of output row y: row_px + j * apitch * 8
                    const size_t row_px = act_off(a.aimg_stride, c.img, y, a.apitch, CO / 8, 0, gx);
                    if constexpr (MODE == CONV_LOGITS_F32 || MODE == CONV_PREDICT) {
                        static_assert(CO == 16, "the logits layer has 16 outputs");
                        if (gx >= a.w) continue;
                        const size_t p = (size_t)c.img * (size_t)a.img_stride + (size_t)y * a.pitch + gx;
#pragma unroll
                        for (int k = 0; k < 16; ++k) v[k] += bias_s[k];
                        if constexpr (MODE == CONV_LOGITS_F32) {
                            float *o = reinterpret_cast<float *>(a.out) + p * a.n_out;
#pragma unroll
                            for (int k = 0; k < 16; ++k)
                                if (k < a.n_out) o[k] = v[k];
                        } else {
                            // argmax of the first n_out logits (ties to the smaller bin; the
                            // logits are finite, the masked bins -inf) as a pairwise tree, then
                            // the softmax probability of the winner: 1 / sum_k exp(v_k - max)
                            float m[16];
                            int ix[16];
#pragma unroll
                            for (int k = 0; k < 16; ++k) {
                                m[k] = v[k];
                                ix[k] = k;
                            }
#pragma unroll
                            for (int st = 1; st < 16; st *= 2)
#pragma unroll
                                for (int k = 0; k < 16; k += 2 * st)
                                    if (m[k + st] > m[k]) {  // the right half wins only when larger
                                        m[k] = m[k + st];
                                        ix[k] = ix[k + st];
                                    }
                            float e[16];
#pragma unroll
                            for (int k = 0; k < 16; ++k) e[k] = __expf(v[k] - m[0]);  // exp(-inf) = 0
#pragma unroll
                            for (int st = 1; st < 16; st *= 2)
#pragma unroll
                                for (int k = 0; k < 16; k += 2 * st) e[k] += e[k + st];
                            a.idx[p] = (uint8_t)ix[0];
                            if (a.conf) a.conf[p] = __frcp_rn(e[0]);
                        }
                    } else {
                        if (gx >= a.apitch) continue;
                        if (gx >= a.w) {  // the zero margin of the activation rows
#pragma unroll
                            for (int k = 0; k < 16; ++k) v[k] = 0.0f;
                        } else if (MODE == CONV_MASK_BF16) {
#pragma unroll
                            for (int h2 = 0; h2 < 2; ++h2) {
                                const uint4 mk = *reinterpret_cast<const uint4 *>(
                                    a.mask + row_px + (size_t)(2 * g + h2) * a.apitch * 8);
                                const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    const uint32_t bits = (mw[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                                    // bf16 > 0: bit patterns 0x0001 .. 0x7F80 (positive, up to +inf)
                                    if (bits - 1u >= 0x7F80u) v[8 * h2 + e] = 0.0f;
                                }
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < 16; ++k) v[k] = fmaxf(v[k] + bias_s[16 * g + k], 0.0f);
                        }
                        __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(a.out);
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            uint4 pk;
                            __nv_bfloat162 b0 = __floats2bfloat162_rn(v[8 * h2 + 0], v[8 * h2 + 1]);
                            __nv_bfloat162 b1 = __floats2bfloat162_rn(v[8 * h2 + 2], v[8 * h2 + 3]);
                            __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * h2 + 4], v[8 * h2 + 5]);
                            __nv_bfloat162 b3 = __floats2bfloat162_rn(v[8 * h2 + 6], v[8 * h2 + 7]);
                            pk.x = *reinterpret_cast<uint32_t *>(&b0);
                            pk.y = *reinterpret_cast<uint32_t *>(&b1);
                            pk.z = *reinterpret_cast<uint32_t *>(&b2);
                            pk.w = *reinterpret_cast<uint32_t *>(&b3);
                            *reinterpret_cast<uint4 *>(ob + row_px + (size_t)(2 * g + h2) * a.apitch * 8) = pk;
                        }
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
    if (tid == 0 && abort_flag && a.status) atomicExch(a.status, FD4_ERR_TIMEOUT);
}


// ---------------------------------------------------------------------------
// Network geometry and the parameter buffer.

constexpr int kLayers = 4;
constexpr int kMaxBins = FD4_SELECTOR_MAX_BINS;  // outputs of the last layer; n_bins of them are used
constexpr int CI_R[kLayers] = {1, 32, 32, 32};   // real channels
constexpr int CO_R[kLayers] = {32, 32, 32, kMaxBins};
constexpr int CI_P[kLayers] = {16, 32, 32, 32};  // padded to the MMA's K and N granularity
constexpr int CO_P[kLayers] = {32, 32, 32, 16};
constexpr int DIL[kLayers] = {1, 2, 4, 8};

struct SelLayout {
    size_t w_off[kLayers], b_off[kLayers];  // master FP32 (floats), order [ky][kx][co][ci]
    size_t n_master;                        // floats per copy (master, m, v, grad)
    size_t fwd_off[kLayers];                // bytes: forward tile layout (bf16)
    size_t dgr_off[kLayers];                // bytes: data-gradient tile layout (layers 1..3)
    size_t bias_off;                        // bytes: padded biases (FP32, CO_P each)
    size_t bytes;
};

SelLayout sel_layout()
{
    SelLayout L{};
    size_t f = 0;
    for (int l = 0; l < kLayers; ++l) {
        L.w_off[l] = f;
        f += (size_t)9 * CO_R[l] * CI_R[l];
        L.b_off[l] = f;
        f += CO_R[l];
    }
    L.n_master = f;
    size_t b = align_up(4 * 4 * f, 256);  // master, m, v, grad
    for (int l = 0; l < kLayers; ++l) {
        L.fwd_off[l] = b;
        b += align_up((size_t)16 * 9 * (CI_P[l] / 8) * CO_P[l], 256);
    }
    for (int l = 1; l < kLayers; ++l) {
        L.dgr_off[l] = b;
        b += align_up((size_t)16 * 9 * (CO_P[l] / 8) * CI_R[l], 256);
    }
    L.bias_off = b;
    b += align_up(sizeof(float) * 32 * kLayers, 256);
    L.bytes = b;
    return L;
}

struct CastArgs {
    const float *master;
    __nv_bfloat16 *fwd[kLayers];
    __nv_bfloat16 *dgr[kLayers];
    float *bias;  // kLayers x 32
    long long w_off[kLayers], b_off[kLayers];
    int ci_p[kLayers], co_p[kLayers], ci_r[kLayers], co_r[kLayers];
};

// Master FP32 weights -> bf16 tile layouts: forward [tap][ci/8][co][8] (zero
// padded) and, for layers 1..3, the data-gradient layout
// [tap'][co/8][ci][8] holding W[8 - tap'][co][ci] (flipped taps, swapped
// channel roles), so the data gradient is the same convolution kernel.
__global__ void k_sel_cast(CastArgs a)
{
    const int l = blockIdx.y;
    const int ci_p = a.ci_p[l], co_p = a.co_p[l], ci_r = a.ci_r[l], co_r = a.co_r[l];
    const float *W = a.master + a.w_off[l];
    const int nf = 9 * ci_p * co_p;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        const int e = i & 7;
        const int co = (i >> 3) % co_p;
        const int j = (i >> 3) / co_p % (ci_p / 8);
        const int t = (i >> 3) / co_p / (ci_p / 8);
        const int ci = 8 * j + e;
        const float v = (co < co_r && ci < ci_r) ? W[((size_t)t * co_r + co) * ci_r + ci] : 0.0f;
        a.fwd[l][i] = __float2bfloat16_rn(v);
    }
    if (l >= 1) {
        const int nd = 9 * co_p * ci_r;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) {
            const int e = i & 7;
            const int c = (i >> 3) % ci_r;              // data-gradient output channel (= forward ci)
            const int j = (i >> 3) / ci_r % (co_p / 8);
            const int t = (i >> 3) / ci_r / (co_p / 8);
            const int k = 8 * j + e;                    // data-gradient input channel (= forward co)
            const float v = k < co_r ? W[((size_t)(8 - t) * co_r + k) * ci_r + c] : 0.0f;
            a.dgr[l][i] = __float2bfloat16_rn(v);
        }
    }
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < 32; c += blockDim.x)
            a.bias[l * 32 + c] = c < co_r ? a.master[a.b_off[l] + c] : 0.0f;
}

// Image -> input activations of layer 0: one stored chunk plane (channel 0 =
// intensity, channels 1..7 = 0; zero from pixel w to the activation pitch);
// the layer reads its second plane (channels 8..15) as zero.
__global__ void k_sel_prep(const float *img, __nv_bfloat16 *act, int n_img, int w, int h, int pitch,
                           long long img_stride, int apitch, long long aimg_stride)
{
    // one block-stride loop over the rows of the stack, threads over columns
    for (int row = blockIdx.x; row < n_img * h; row += gridDim.x) {
        const int i = row / h, y = row - (row / h) * h;
        const size_t base = (size_t)i * (size_t)img_stride + (size_t)y * pitch;
        for (int x = threadIdx.x; x < apitch; x += blockDim.x) {
            __nv_bfloat162 b = __floats2bfloat162_rn(x < w ? img[base + x] : 0.0f, 0.0f);
            *reinterpret_cast<uint4 *>(act + act_off(aimg_stride, i, y, apitch, 1, 0, x)) =
                make_uint4(*reinterpret_cast<uint32_t *>(&b), 0u, 0u, 0u);
        }
    }
}

// Softmax cross-entropy over the n_bins logits of every pixel (n_bins floats
// per pixel): mean loss added to *loss, gradient (p - onehot) / npx written as
// row-planar bf16 (16 channels, those from n_bins on zero; zero from pixel w
// to the activation pitch).
__global__ void __launch_bounds__(256) k_sel_softmax_ce(const float *logits, const uint8_t *labels,
                                                        __nv_bfloat16 *dz, int n_img, int w, int h, int pitch,
                                                        long long img_stride, int apitch, long long aimg_stride,
                                                        float inv_npx, float *loss, int n_bins)
{
    __shared__ float red[8];
    float lsum = 0.0f;
    for (int row = blockIdx.x; row < n_img * h; row += gridDim.x)
    for (int x = threadIdx.x; x < apitch; x += blockDim.x) {
        const size_t i = (size_t)(row / h) * (size_t)img_stride + (size_t)(row % h) * pitch + x;
        float g[kMaxBins];
#pragma unroll
        for (int c = 0; c < kMaxBins; ++c) g[c] = 0.0f;
        if (x < w) {
            const float *z = logits + i * n_bins;
            float m = z[0];
            for (int c = 1; c < n_bins; ++c) m = fmaxf(m, z[c]);
            float sum = 0.0f;
#pragma unroll
            for (int c = 0; c < kMaxBins; ++c)
                if (c < n_bins) {
                    g[c] = expf(z[c] - m);
                    sum += g[c];
                }
            const int lab = labels[i] < n_bins ? labels[i] : n_bins - 1;
            lsum += logf(sum) - (z[lab] - m);
#pragma unroll
            for (int c = 0; c < kMaxBins; ++c)
                if (c < n_bins) g[c] = (g[c] / sum - (c == lab ? 1.0f : 0.0f)) * inv_npx;
        }
        uint32_t q[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            __nv_bfloat162 b = __floats2bfloat162_rn(g[2 * c], g[2 * c + 1]);
            q[c] = *reinterpret_cast<uint32_t *>(&b);
        }
        const int im = row / h, y = row - (row / h) * h;
        *reinterpret_cast<uint4 *>(dz + act_off(aimg_stride, im, y, apitch, 2, 0, x)) = make_uint4(q[0], q[1], q[2], q[3]);
        *reinterpret_cast<uint4 *>(dz + act_off(aimg_stride, im, y, apitch, 2, 1, x)) = make_uint4(q[4], q[5], q[6], q[7]);
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        atomicAdd(loss, s * inv_npx);
    }
}

// Weight gradient of one layer on the tensor cores:
//   gW[t][co][ci] += sum_px dZ[px][co] X[px + shift_t][ci],  gb[co] += sum_px dZ[px][co],
// as the product D[m][n] = sum_k A[m][k] B[n][k] over the pixels k of a
// 128-pixel row tile (the MMA's K, 16 per instruction): A's rows m are the
// output channels (COP of the 128 rows; the rest stay zero), B's rows n are
// the tap-shifted inputs n = t CIP + ci, then a row of ones whose product is
// the bias gradient, then zero rows up to a multiple of 16.  Both operands
// are K-major without swizzle (8 x 16-byte core matrices: LBO 128 bytes
// along K, SBO 2048 bytes along M / N).  A persistent block accumulates all
// its tiles in tensor memory (lane = output channel, column = n) and adds the
// sums to gW and gb once at the end.
template <int CIP>
constexpr int wg_rows() { return 9 * CIP + 16; }
template <int CIP>
constexpr size_t wg_smem()
{
    return 1024 + (size_t)2 * 128 * TM + (size_t)2 * wg_rows<CIP>() * TM + (size_t)2 * 3 * (TM + 2 * kMaxDil) * CIP;
}

__device__ __forceinline__ uint32_t wg_off(int row, int k)  // byte offset of element (row, k), K-major core layout
{
    return (uint32_t)((row >> 3) * 2048 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int CIP, int COP>
__global__ void __launch_bounds__(CT, 1)
    k_sel_wgrad_tc(const __nv_bfloat16 *X, int x_cj, const __nv_bfloat16 *dZ, int ci_r, int co_r, int n_img, int w,
                   int h, int apitch, int d, long long aimg_stride, float *gW, float *gb, int *status)
{
    constexpr int NB = wg_rows<CIP>(), CJ = CIP / 8;
    constexpr int N0 = NB > 256 ? ((NB / 2 + 15) / 16) * 16 : NB;  // first chunk of B rows (MMA N <= 256)
    constexpr int N1 = NB - N0;
    static_assert(N0 % 16 == 0 && N1 % 16 == 0 && N0 <= 256 && N1 <= 256, "MMA N of M = 128");
    extern __shared__ unsigned char wg_raw[];
    unsigned char *As = reinterpret_cast<unsigned char *>(((uintptr_t)wg_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Bs = As + 2 * 128 * TM;
    __nv_bfloat16 *Xs = reinterpret_cast<__nv_bfloat16 *>(Bs + 2 * NB * TM);  // [3][P][CIP]
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = TM + 2 * d;
    // A: all zero (rows from COP on stay so); B: the ones row and the zero rows after it
    for (int i = tid; i < 128 * TM * 2 / 16; i += CT) reinterpret_cast<uint4 *>(As)[i] = make_uint4(0u, 0u, 0u, 0u);
    {
        const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
        for (int i = tid; i < (NB - 9 * CIP) * TM; i += CT) {
            const int row = 9 * CIP + i / TM, k = i % TM;
            *reinterpret_cast<__nv_bfloat16 *>(Bs + wg_off(row, k)) = row == 9 * CIP ? one : zero;
        }
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        abort_flag = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const int tiles_x = (w + TM - 1) / TM;
    const long long total = (long long)n_img * h * tiles_x;
    uint32_t phase = 0;
    bool any = false;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int tx = (int)(t % tiles_x);
        const long long rr = t / tiles_x;
        const int y = (int)(rr % h);
        const int img = (int)(rr / h);
        const int x0 = tx * TM;
        // X rows y - d, y, y + d; pixels x0 - d .. x0 + TM - 1 + d (zero outside the
        // image and in the chunk planes X does not store)
        for (int ky = 0; ky < 3; ++ky) {
            const int gy = y + (ky - 1) * d;
            const bool row_in = gy >= 0 && gy < h;
            for (int e = tid; e < P * CJ; e += CT) {
                const int j = e / P, p = e - (e / P) * P;  // consecutive threads read consecutive pixels
                const int gx = x0 - d + p;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (row_in && j < x_cj && gx >= 0 && gx < w)
                    v = *reinterpret_cast<const uint4 *>(X + act_off(aimg_stride, img, gy, apitch, x_cj, j, gx));
                *reinterpret_cast<uint4 *>(Xs + ((size_t)ky * P + p) * CIP + 8 * j) = v;
            }
        }
        // A rows co < COP: dZ of the tile's pixels (zero beyond the image)
        for (int e = tid; e < TM * (COP / 8); e += CT) {
            const int k = e % TM, g = e / TM;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (x0 + k < w)
                v = *reinterpret_cast<const uint4 *>(dZ + act_off(aimg_stride, img, y, apitch, COP / 8, g, x0 + k));
            const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
                *reinterpret_cast<unsigned short *>(As + wg_off(8 * g + r, k)) =
                    (unsigned short)(vw[r >> 1] >> (16 * (r & 1)));
        }
        __syncthreads();  // Xs is complete
        // B rows n = t CIP + ci: core matrix (8 channels x 8 pixels) from 8 pixel chunks
        for (int e = tid; e < (9 * CJ) * (TM / 8); e += CT) {
            const int kg = e % (TM / 8), ng = e / (TM / 8);
            const int tap = ng / CJ, j = ng % CJ, ky = tap / 3, kx = tap % 3;
            uint4 px[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                px[q] = *reinterpret_cast<const uint4 *>(Xs + ((size_t)ky * P + 8 * kg + q + kx * d) * CIP + 8 * j);
            // channel c of pixel q: half (c % 2) of word c / 2 of px[q]; row c of the
            // core matrix packs pixels (2i, 2i + 1) into word i
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const unsigned sel = (c & 1) ? 0x7632u : 0x5410u;
                uint32_t wq[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    wq[q] = (c >> 1) == 0 ? px[q].x : (c >> 1) == 1 ? px[q].y : (c >> 1) == 2 ? px[q].z : px[q].w;
                uint4 row;
                row.x = __byte_perm(wq[0], wq[1], sel);
                row.y = __byte_perm(wq[2], wq[3], sel);
                row.z = __byte_perm(wq[4], wq[5], sel);
                row.w = __byte_perm(wq[6], wq[7], sel);
                *reinterpret_cast<uint4 *>(Bs + wg_off(8 * ng + c, 8 * kg)) = row;
            }
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
#pragma unroll 1
            for (int ks = 0; ks < TM / 16; ++ks) {
                const uint32_t acc = (any || ks > 0) ? 1u : 0u;
                const uint64_t ad = tc::sdesc_kmajor(a0 + ks * 256, 128, 2048);
                tc::mma_bf16(tmem, ad, tc::sdesc_kmajor(b0 + ks * 256, 128, 2048), tc::idesc_bf16_f32(128, N0), acc);
                if (N1 > 0)
                    tc::mma_bf16(tmem + N0, ad, tc::sdesc_kmajor(b0 + (N0 / 8) * 2048 + ks * 256, 128, 2048),
                                 tc::idesc_bf16_f32(128, N1), acc);
            }
            tc::mma_commit(&mbar);
        }
        any = true;
        {  // the MMAs have read the operands before they are restaged: at most one second
            const uint64_t t0 = globaltimer();
            while (!tc::mbar_try_wait(&mbar, phase)) {
                if (globaltimer() - t0 > 1000000000ull) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
            }
        }
        phase ^= 1u;
        tc::fence_after_sync();
        __syncthreads();
        if (abort_flag) break;
    }
    // the sums: warp 0's lanes are the output channels
    if (any && !abort_flag && warp == 0) {
#pragma unroll 1
        for (int cb = 0; cb < (NB + 31) / 32; ++cb) {
            float v[32];
            tc::tmem_ld_x32(tmem + (uint32_t)(cb * 32), v);
            if (lane < co_r) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int n = cb * 32 + i;
                    if (n < 9 * CIP) {
                        const int tap = n / CIP, ci = n - tap * CIP;
                        if (ci < ci_r) atomicAdd(gW + ((size_t)tap * co_r + lane) * ci_r + ci, v[i]);
                    } else if (n == 9 * CIP) {
                        atomicAdd(gb + lane, v[i]);
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if (tid == 0 && abort_flag && status) atomicExch(status, FD4_ERR_TIMEOUT);
}

// Adam on the FP32 master weights; the gradient is cleared afterwards.
__global__ void k_sel_adam(float *w, float *m, float *v, float *g, size_t n, float lr, float b1, float b2, float eps,
                           float c1, float c2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        g[i] = 0.0f;
    }
}

// Tiles (32 x 64, the scale sweep's tiling) whose least confident pixel is
// below thr go to the fallback list.
__global__ void __launch_bounds__(256) k_sel_fallback_tiles(const float *conf, int w, int h, int pitch, float thr,
                                                            int *list, int *count)
{
    __shared__ float red[8];
    const int tiles_x = (w + 31) / 32;
    const int t = blockIdx.x;
    const int x0 = (t % tiles_x) * 32, y0 = (t / tiles_x) * 64;
    float m = 1.0f;
    for (int i = threadIdx.x; i < 32 * 64; i += 256) {
        const int x = x0 + (i & 31), y = y0 + (i >> 5);
        if (x < w && y < h) m = fminf(m, conf[(size_t)y * pitch + x]);
    }
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < 8; ++i) m = fminf(m, red[i]);
        m = fminf(m, red[0]);
        if (m < thr) list[atomicAdd(count, 1)] = t;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side.

namespace {

// Persistent grid of a kernel that allocates `cols` TMEM columns per block.
// The runtime's occupancy query reports one block per SM for any kernel that
// uses tcgen05.alloc, whatever its resources, so the blocks per SM are taken
// here from registers and shared memory, and capped so that every resident
// block's columns fit the SM's 512 (an allocation never waits on another block).
int tmem_grid(const void *kernel, size_t dyn_smem, int tiles, int cols, int threads = CT)
{
    static int sms = 0, regs_sm = 0, smem_sm = 0, smem_reserved = 0;
    int dev = 0;
    if (sms == 0) {
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
            sms = 0;
            return tiles < 152 ? (tiles > 0 ? tiles : 1) : 152;
        }
    }
    cudaFuncAttributes fa;
    int per_sm = 1;
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) {
        const int warps = (threads + 31) / 32;
        const int regs_block = warps * ((fa.numRegs * 32 + 255) / 256) * 256;
        const size_t smem_block = fa.sharedSizeBytes + dyn_smem + (size_t)smem_reserved;
        per_sm = regs_block > 0 ? regs_sm / regs_block : 1;
        if (smem_block > 0) per_sm = std::min<int>(per_sm, (int)((size_t)smem_sm / smem_block));
        per_sm = std::min(per_sm, std::min(2048 / threads, 512 / cols));
        if (per_sm < 1) per_sm = 1;
    }
    const long long g = (long long)per_sm * sms;
    return (int)(tiles < g ? (tiles > 0 ? tiles : 1) : g);
}

// Tensor map of a row-planar activation tensor in 8-pixel segments (16
// elements of 8 bytes = 128 bytes of one chunk plane): dimensions {16,
// apitch / 8 segments, cj stored chunk planes, h rows, n_img images}; box
// {16, 18, cj, 1, 1}, a 144-pixel window of a row in every stored plane.
// Segments outside the row and rows outside 0 .. h - 1 read as zero; the
// pixels w .. apitch - 1 are zero in memory.
int make_act_map(CUtensorMap *m, const void *act, int cj, int apitch, int h, long long aimg_stride, int n_img)
{
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)act & 15u) || apitch % kSegPx) return 1;
    const cuuint64_t dim[5] = {16, (cuuint64_t)apitch / kSegPx, (cuuint64_t)cj, (cuuint64_t)h, (cuuint64_t)n_img};
    const cuuint64_t str[4] = {128, (cuuint64_t)apitch * 16, (cuuint64_t)apitch * cj * 16,
                               (cuuint64_t)aimg_stride * cj * 16};
    const cuuint32_t box[5] = {16, kWinPx / kSegPx, (cuuint32_t)cj, 1, 1};
    const cuuint32_t one[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void *>(act), dim, str, box, one,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS;
}

template <int CI, int CO, int MODE>
int launch_conv(const ConvArgs &a, cudaStream_t st)
{
    const size_t smem = conv_smem_bytes(CI, CO);
    static int attr_dev = -1;
    int dev = 0;
    if (a.d < 1 || a.d > kMaxDil || a.in_cj < 1 || a.in_cj > CI / 8 || a.apitch != act_pitch(a.w)) return 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (attr_dev != dev) {
        if (cudaFuncSetAttribute(k_conv_tc<CI, CO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 1;
        attr_dev = dev;
    }
    CUtensorMap map;
    if (make_act_map(&map, a.in, a.in_cj, a.apitch, a.h, a.aimg_stride, a.n_img)) return 1;
    // Segment length: about four units per resident block (each unit reads
    // two input rows more than it writes; long segments leave blocks idle),
    // 4 .. 64 rows.
    const int resident =
        tmem_grid((const void *)k_conv_tc<CI, CO, MODE>, smem, 1 << 30, (int)conv_tmem_cols(CO), conv_threads(CO));
    const long long tiles = (long long)a.n_img * a.h * ((a.w + TM - 1) / TM);
    ConvArgs b = a;
    b.seg_rows = (int)std::max<long long>(4, std::min<long long>(64, tiles / (4LL * resident)));
    const long long units = conv_units(b.n_img, b.w, b.h, b.d, b.seg_rows);
    const int grid = (int)std::min<long long>(units, resident);
    k_conv_tc<CI, CO, MODE><<<grid, conv_threads(CO), smem, st>>>(map, b);
    return cudaGetLastError() != cudaSuccess;
}

struct SelBufs {
    __nv_bfloat16 *act[kLayers];  // inputs of layers 0..3, row-planar (8 stored / 32 / 32 / 32 channels)
    float *logits;                // n_bins per pixel (room for kMaxBins)
    __nv_bfloat16 *dz16;          // gradient of the last layer's output (16 channels)
    __nv_bfloat16 *dz[2];         // 32-channel gradients (ping-pong)
    int *status;
    size_t bytes;
};

// Workspace of the network for a stack of n_img images (h rows; the
// activations at act_pitch(w) pixels per row, the logits at `pitch`).
// Training keeps every layer's input for the backward pass; inference (infer)
// needs the input of the current layer only, so layers 1 and 3 share one
// buffer: [status | act0 | A | B | logits], with act1 = act3 = A and act2 = B.
SelBufs sel_bufs(char *ws, int n_img, int w, int h, int pitch, bool infer = false)
{
    SelBufs b{};
    const long long npx = (long long)n_img * h * act_pitch(w);  // activation pixels
    const long long lpx = (long long)n_img * h * pitch;         // logit pixels
    size_t o = 256;  // header: status word
    b.status = (int *)ws;
    const size_t per[kLayers] = {8, 32, 32, 32};  // layer 0 stores one chunk plane of its 16 channels
    for (int l = 0; l < kLayers; ++l) {
        if (infer && l == 3) {
            b.act[3] = b.act[1];
            continue;
        }
        b.act[l] = ws ? (__nv_bfloat16 *)(ws + o) : nullptr;
        o += align_up((size_t)npx * per[l] * 2, 256);
    }
    b.logits = ws ? (float *)(ws + o) : nullptr;
    o += align_up((size_t)lpx * kMaxBins * 4, 256);
    if (infer) {
        b.bytes = o;
        return b;
    }
    b.dz16 = ws ? (__nv_bfloat16 *)(ws + o) : nullptr;
    o += align_up((size_t)npx * 16 * 2, 256);
    for (int k = 0; k < 2; ++k) {
        b.dz[k] = ws ? (__nv_bfloat16 *)(ws + o) : nullptr;
        o += align_up((size_t)npx * 32 * 2, 256);
    }
    b.bytes = o;
    return b;
}

struct SelPtrs {
    float *master, *m, *v, *grad;
    const uint4 *fwd[kLayers];
    const uint4 *dgr[kLayers];
    const float *bias;
};

SelPtrs sel_ptrs(void *params)
{
    const SelLayout L = sel_layout();
    char *p = (char *)params;
    SelPtrs s{};
    s.master = (float *)p;
    s.m = s.master + L.n_master;
    s.v = s.m + L.n_master;
    s.grad = s.v + L.n_master;
    for (int l = 0; l < kLayers; ++l) s.fwd[l] = (const uint4 *)(p + L.fwd_off[l]);
    for (int l = 1; l < kLayers; ++l) s.dgr[l] = (const uint4 *)(p + L.dgr_off[l]);
    s.bias = (const float *)(p + L.bias_off);
    return s;
}

int sel_recast(void *params, cudaStream_t st)
{
    const SelLayout L = sel_layout();
    char *p = (char *)params;
    CastArgs a{};
    a.master = (const float *)p;
    for (int l = 0; l < kLayers; ++l) {
        a.fwd[l] = (__nv_bfloat16 *)(p + L.fwd_off[l]);
        a.dgr[l] = l ? (__nv_bfloat16 *)(p + L.dgr_off[l]) : nullptr;
        a.w_off[l] = (long long)L.w_off[l];
        a.b_off[l] = (long long)L.b_off[l];
        a.ci_p[l] = CI_P[l];
        a.co_p[l] = CO_P[l];
        a.ci_r[l] = CI_R[l];
        a.co_r[l] = CO_R[l];
    }
    a.bias = (float *)(p + L.bias_off);
    k_sel_cast<<<dim3(16, kLayers), 256, 0, st>>>(a);
    return cudaGetLastError() != cudaSuccess;
}

int check_stack(const void *d, int n_img, int w, int h, int pitch)
{
    if (n_img < 1) return FD4_ERR_BAD_ARG;
    return check_image(d, w, h, pitch);
}

// Forward pass of the network over a stack of n_img images (img_stride = h * pitch).
// Geometry fields of a convolution over a stack of n_img images.
ConvArgs conv_geometry(int n_img, int w, int h, int pitch, int *status)
{
    ConvArgs a{};
    a.n_img = n_img;
    a.w = w;
    a.h = h;
    a.pitch = pitch;
    a.apitch = act_pitch(w);
    a.img_stride = (long long)h * pitch;
    a.aimg_stride = (long long)h * a.apitch;
    a.status = status;
    return a;
}

// With idx set, the last layer writes the prediction (argmax bin and its
// probability) instead of the logits.
int sel_forward(const SelPtrs &P, const float *imgs, int n_img, int w, int h, int pitch, int n_bins,
                const SelBufs &B, cudaStream_t st, uint8_t *idx = nullptr, float *conf = nullptr)
{
    const ConvArgs g0 = conv_geometry(n_img, w, h, pitch, B.status);
    const int g = n_img * h < 8192 ? n_img * h : 8192;  // blocks stride over image rows
    k_sel_prep<<<g, 256, 0, st>>>(imgs, B.act[0], n_img, w, h, pitch, g0.img_stride, g0.apitch, g0.aimg_stride);
    ConvArgs a = g0;
    for (int l = 0; l < kLayers; ++l) {
        a.in = B.act[l];
        a.in_cj = l == 0 ? 1 : CI_P[l] / 8;
        a.wts = P.fwd[l];
        a.bias = P.bias + 32 * l;
        a.d = DIL[l];
        a.mask = nullptr;
        int rc;
        if (l == 0) {
            a.out = B.act[1];
            rc = launch_conv<16, 32, CONV_RELU_BF16>(a, st);
        } else if (l < kLayers - 1) {
            a.out = B.act[l + 1];
            rc = launch_conv<32, 32, CONV_RELU_BF16>(a, st);
        } else if (idx) {
            a.out = nullptr;
            a.idx = idx;
            a.conf = conf;
            a.n_out = n_bins;
            rc = launch_conv<32, 16, CONV_PREDICT>(a, st);
        } else {
            a.out = B.logits;
            a.n_out = n_bins;
            rc = launch_conv<32, 16, CONV_LOGITS_F32>(a, st);
        }
        if (rc) return 1;
    }
    return 0;
}

template <int CIP, int COP>
int launch_wgrad(const __nv_bfloat16 *X, const __nv_bfloat16 *dZ, int l, const SelPtrs &P, int n_img, int w, int h,
                 int *status, cudaStream_t st)
{
    const SelLayout L = sel_layout();
    static int attr_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (attr_dev != dev) {
        if (cudaFuncSetAttribute(k_sel_wgrad_tc<CIP, COP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wg_smem<CIP>()) != cudaSuccess)
            return 1;
        attr_dev = dev;
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (long long)n_img * h * ((w + TM - 1) / TM);
    const int grid = (int)(tiles < sms ? (tiles > 0 ? tiles : 1) : sms);  // one block (all of TMEM) per SM
    const int apitch = act_pitch(w);
    k_sel_wgrad_tc<CIP, COP><<<grid, CT, wg_smem<CIP>(), st>>>(X, l == 0 ? 1 : CIP / 8, dZ, CI_R[l], CO_R[l], n_img,
                                                               w, h, apitch, DIL[l], (long long)h * apitch,
                                                               P.grad + L.w_off[l], P.grad + L.b_off[l], status);
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace
}  // namespace fd4

using namespace fd4;

extern "C" size_t fd4_selector_param_bytes(void) { return sel_layout().bytes; }

extern "C" size_t fd4_selector_workspace_bytes(int n_img, int w, int h, int pitch)
{
    if (n_img < 1 || w < 1 || h < 1 || pitch < w) return 0;
    return sel_bufs(nullptr, n_img, w, h, pitch).bytes;
}

extern "C" size_t fd4_selector_infer_workspace_bytes(int n_img, int w, int h, int pitch)
{
    if (n_img < 1 || w < 1 || h < 1 || pitch < w) return 0;
    return sel_bufs(nullptr, n_img, w, h, pitch, true).bytes;
}

extern "C" int fd4_selector_set_weights(void *d_params, const float *h_w, fd4_stream_t stream)
{
    if (!d_params || !h_w || ((uintptr_t)d_params & 255u)) return FD4_ERR_BAD_ARG;
    const SelLayout L = sel_layout();
    cudaStream_t st = (cudaStream_t)stream;
    // master weights from the host; moments and gradients cleared
    if (cudaMemcpyAsync(d_params, h_w, sizeof(float) * L.n_master, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FD4_ERR_CUDA;
    if (cudaMemsetAsync((float *)d_params + L.n_master, 0, sizeof(float) * 3 * L.n_master, st) != cudaSuccess)
        return FD4_ERR_CUDA;
    if (sel_recast(d_params, st)) return FD4_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? FD4_OK : FD4_ERR_CUDA;
}

extern "C" int fd4_selector_get_weights(const void *d_params, float *h_w, int which, fd4_stream_t stream)
{
    if (!d_params || !h_w || which < 0 || which > 3) return FD4_ERR_BAD_ARG;
    const SelLayout L = sel_layout();
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(h_w, (const float *)d_params + (size_t)which * L.n_master, sizeof(float) * L.n_master,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FD4_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? FD4_OK : FD4_ERR_CUDA;
}

extern "C" int fd4_selector_init(void *d_params, unsigned long long seed, fd4_stream_t stream)
{
    // He-normal initialisation on the host (SplitMix64 + Box-Muller), biases 0
    const SelLayout L = sel_layout();
    float *h = new float[L.n_master]();
    unsigned long long state = seed;
    auto next = [&state]() {
        unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto unif = [&next]() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    for (int l = 0; l < kLayers; ++l) {
        const double std = sqrt(2.0 / (9.0 * CI_R[l]));
        const size_t n = (size_t)9 * CO_R[l] * CI_R[l];
        for (size_t i = 0; i < n; ++i) {
            const double u1 = unif(), u2 = unif();
            h[L.w_off[l] + i] = (float)(std * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
        }
    }
    const int rc = fd4_selector_set_weights(d_params, h, stream);
    delete[] h;
    return rc;
}

static bool bins_ok(int n_bins) { return n_bins >= 2 && n_bins <= kMaxBins; }

extern "C" int fd4_selector_forward(const void *d_params, const float *d_imgs, int n_img, int w, int h, int pitch,
                                    int n_bins, float *d_logits, void *d_ws, size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    if (!d_params || !d_logits || !bins_ok(n_bins)) return FD4_ERR_BAD_ARG;
    if ((rc = check_stack(d_imgs, n_img, w, h, pitch)) != FD4_OK) return rc;
    const long long npx = (long long)n_img * h * pitch;
    if (!d_ws || ws_bytes < fd4_selector_infer_workspace_bytes(n_img, w, h, pitch)) return FD4_ERR_WS_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    SelBufs B = sel_bufs((char *)d_ws, n_img, w, h, pitch, true);
    if (cudaMemsetAsync(B.status, 0, sizeof(int), st) != cudaSuccess) return FD4_ERR_CUDA;
    if (sel_forward(sel_ptrs((void *)d_params), d_imgs, n_img, w, h, pitch, n_bins, B, st)) return FD4_ERR_CUDA;
    if (cudaMemcpyAsync(d_logits, B.logits, sizeof(float) * n_bins * npx, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return FD4_ERR_CUDA;
    return FD4_OK;
}

extern "C" int fd4_selector_grad(void *d_params, const float *d_imgs, const uint8_t *d_labels, int n_img, int w,
                                 int h, int pitch, int n_bins, float *d_loss, void *d_ws, size_t ws_bytes,
                                 fd4_stream_t stream)
{
    int rc;
    if (!d_params || !d_labels || !d_loss || !bins_ok(n_bins)) return FD4_ERR_BAD_ARG;
    if ((rc = check_stack(d_imgs, n_img, w, h, pitch)) != FD4_OK) return rc;
    if (!d_ws || ws_bytes < fd4_selector_workspace_bytes(n_img, w, h, pitch)) return FD4_ERR_WS_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    SelBufs B = sel_bufs((char *)d_ws, n_img, w, h, pitch);
    const SelPtrs P = sel_ptrs(d_params);
    if (cudaMemsetAsync(B.status, 0, sizeof(int), st) != cudaSuccess) return FD4_ERR_CUDA;
    if (sel_forward(P, d_imgs, n_img, w, h, pitch, n_bins, B, st)) return FD4_ERR_CUDA;
    ConvArgs a = conv_geometry(n_img, w, h, pitch, B.status);
    const int g = n_img * h < 8192 ? n_img * h : 8192;
    k_sel_softmax_ce<<<g, 256, 0, st>>>(B.logits, d_labels, B.dz16, n_img, w, h, pitch, a.img_stride, a.apitch,
                                        a.aimg_stride, 1.0f / (float)((long long)n_img * w * h), d_loss, n_bins);
    // layer 3 (last): weight gradient, then data gradient into dz[0] masked by act[3] > 0
    if (launch_wgrad<32, 16>(B.act[3], B.dz16, 3, P, n_img, w, h, B.status, st)) return FD4_ERR_CUDA;
    a.in = B.dz16;
    a.in_cj = 2;
    a.out = B.dz[0];
    a.wts = P.dgr[3];
    a.bias = nullptr;
    a.mask = B.act[3];
    a.d = DIL[3];
    if (launch_conv<16, 32, CONV_MASK_BF16>(a, st)) return FD4_ERR_CUDA;
    int cur = 0;
    for (int l = 2; l >= 1; --l) {
        if (launch_wgrad<32, 32>(B.act[l], B.dz[cur], l, P, n_img, w, h, B.status, st)) return FD4_ERR_CUDA;
        a.in = B.dz[cur];
        a.in_cj = 4;
        a.out = B.dz[cur ^ 1];
        a.wts = P.dgr[l];
        a.mask = B.act[l];
        a.d = DIL[l];
        if (launch_conv<32, 32, CONV_MASK_BF16>(a, st)) return FD4_ERR_CUDA;
        cur ^= 1;
    }
    if (launch_wgrad<16, 32>(B.act[0], B.dz[cur], 0, P, n_img, w, h, B.status, st)) return FD4_ERR_CUDA;
    return FD4_OK;
}

extern "C" int fd4_selector_update(void *d_params, float lr, int step, fd4_stream_t stream)
{
    if (!d_params || step < 1 || !(lr > 0.0f)) return FD4_ERR_BAD_ARG;
    const SelLayout L = sel_layout();
    const SelPtrs P = sel_ptrs(d_params);
    cudaStream_t st = (cudaStream_t)stream;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - pow(0.9, step)), c2 = (float)(1.0 - pow(0.999, step));
    k_sel_adam<<<64, 256, 0, st>>>(P.master, P.m, P.v, P.grad, L.n_master, lr, b1, b2, 1e-8f, c1, c2);
    if (sel_recast(d_params, st)) return FD4_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? FD4_OK : FD4_ERR_CUDA;
}

extern "C" int fd4_selector_predict(const void *d_params, const float *d_imgs, int n_img, int w, int h, int pitch,
                                    int n_bins, uint8_t *d_idx, float *d_conf, void *d_ws, size_t ws_bytes,
                                    fd4_stream_t stream)
{
    int rc;
    if (!d_params || !d_idx || !bins_ok(n_bins)) return FD4_ERR_BAD_ARG;
    if ((rc = check_stack(d_imgs, n_img, w, h, pitch)) != FD4_OK) return rc;
    if (!d_ws || ws_bytes < fd4_selector_infer_workspace_bytes(n_img, w, h, pitch)) return FD4_ERR_WS_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    SelBufs B = sel_bufs((char *)d_ws, n_img, w, h, pitch, true);
    if (cudaMemsetAsync(B.status, 0, sizeof(int), st) != cudaSuccess) return FD4_ERR_CUDA;
    if (sel_forward(sel_ptrs((void *)d_params), d_imgs, n_img, w, h, pitch, n_bins, B, st, d_idx, d_conf))
        return FD4_ERR_CUDA;
    return FD4_OK;
}

extern "C" int fd4_selector_status(const void *d_ws, int *status, fd4_stream_t stream)
{
    if (!d_ws || !status) return FD4_ERR_BAD_ARG;
    if (cudaMemcpyAsync(status, d_ws, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return FD4_ERR_CUDA;
    return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? FD4_OK : FD4_ERR_CUDA;
}

// Learned selection with the plain selection as fallback.
// Workspace: [selector buffers | confidence plane | selection workspace | tile list].
static size_t learned_parts(int w, int h, int pitch, int n_sigma, size_t *o_conf, size_t *o_sel, size_t *o_list)
{
    size_t o = align_up(fd4_selector_infer_workspace_bytes(1, w, h, pitch), 256);
    *o_conf = o;
    o += align_up((size_t)h * pitch * sizeof(float), 256);
    *o_sel = o;
    o += ws_select_bytes(h, pitch, n_sigma);
    *o_list = o;
    const int tiles = ((w + 31) / 32) * ((h + 63) / 64);
    o += align_up(sizeof(int) * ((size_t)tiles + 1), 256);
    return o;
}

extern "C" size_t fd4_select_learned_workspace_bytes(int w, int h, int pitch, int n_sigma)
{
    if (w < 1 || h < 1 || pitch < w || n_sigma < 1) return 0;
    size_t a, b, c;
    return learned_parts(w, h, pitch, n_sigma, &a, &b, &c);
}

extern "C" int fd4_select_scales_learned(const void *d_params, const float *d_img, int w, int h, int pitch,
                                         const float *h_sigmas, int n_sigma, const fd4_params *params,
                                         float conf_threshold, uint8_t *d_sigma_idx, float *d_conf,
                                         int *d_n_fallback, void *d_ws, size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    fd4_params p;
    resolve_params(params, &p);
    if (!d_params || !d_sigma_idx) return FD4_ERR_BAD_ARG;
    if ((rc = check_image(d_img, w, h, pitch)) != FD4_OK) return rc;
    if ((rc = check_sigmas(h_sigmas, n_sigma)) != FD4_OK) return rc;
    if (!bins_ok(n_sigma)) return FD4_ERR_BAD_ARG;  // one bin per scale, at most kMaxBins
    if (!(conf_threshold >= 0.0f && conf_threshold <= 1.0f)) return FD4_ERR_BAD_ARG;
    size_t o_conf, o_sel, o_list;
    const size_t need = learned_parts(w, h, pitch, n_sigma, &o_conf, &o_sel, &o_list);
    if (!d_ws || ((uintptr_t)d_ws & 255u)) return FD4_ERR_BAD_ARG;
    if (ws_bytes < need) return FD4_ERR_WS_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    float *conf = (float *)(ws + o_conf);
    char *sel = ws + o_sel;
    int *list = (int *)(ws + o_list);
    const int tiles = ((w + 31) / 32) * ((h + 63) / 64);
    int *count = list + tiles;
    if ((rc = fd4_selector_predict(d_params, d_img, 1, w, h, pitch, n_sigma, d_sigma_idx, conf, d_ws, ws_bytes,
                                   stream)) != FD4_OK)
        return rc;
    if (cudaMemsetAsync(count, 0, sizeof(int), st) != cudaSuccess) return FD4_ERR_CUDA;
    k_sel_fallback_tiles<<<tiles, 256, 0, st>>>(conf, w, h, pitch, conf_threshold, list, count);
    // plain selection on the listed tiles, overwriting the prediction there
    const size_t pb = plane_bytes(h, pitch, 4);
    ImgDesc d{};
    d.in = d_img;
    d.vp = (float *)(sel + kHeaderBytes);
    d.s2 = (float *)(sel + kHeaderBytes + (size_t)n_sigma * pb);
    d.plane = pb / 4;
    d.idx = d_sigma_idx;
    d.max_s2 = &((WsHeader *)sel)->max_s2;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    if (launch_select_tiles(d, list, count, h_sigmas, n_sigma, p, st)) return FD4_ERR_CUDA;
    if (d_conf && cudaMemcpyAsync(d_conf, conf, sizeof(float) * (size_t)h * pitch, cudaMemcpyDeviceToDevice, st) !=
                      cudaSuccess)
        return FD4_ERR_CUDA;
    if (d_n_fallback &&
        cudaMemcpyAsync(d_n_fallback, count, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return FD4_ERR_CUDA;
    return FD4_OK;
}

extern "C" int fd4_selftest_wait_timeout(void *d_ws, size_t ws_bytes, int *status, fd4_stream_t stream)
{
    const int w = 128, h = 4, pitch = 128;
    if (!d_ws || !status || ((uintptr_t)d_ws & 255u)) return FD4_ERR_BAD_ARG;
    if (ws_bytes < fd4_selector_workspace_bytes(1, w, h, pitch)) return FD4_ERR_WS_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    SelBufs B = sel_bufs((char *)d_ws, 1, w, h, pitch);
    if (cudaMemsetAsync(d_ws, 0, fd4_selector_workspace_bytes(1, w, h, pitch), st) != cudaSuccess)
        return FD4_ERR_CUDA;
    ConvArgs a = conv_geometry(1, w, h, pitch, B.status);
    a.in = B.act[1];
    a.in_cj = 4;
    a.out = B.act[2];
    a.wts = (const uint4 *)B.act[3];  // zeros; never multiplied
    a.d = 1;
    a.withhold_commit = 1;
    if (launch_conv<32, 32, CONV_RELU_BF16>(a, st)) return FD4_ERR_CUDA;
    return fd4_selector_status(d_ws, status, stream);
}
