// Derivatives of u_sigma at each pixel's selected scale for the tensor build
// (Sec. 3.3 Eq. 9: N = H(u_sigma*) / sqrt(1 + |grad u_sigma*|), the normalised
// Hessian before its G_rho smoothing).
//
// One launch per scale of the set.  A block takes a strip segment (32 columns
// x 512 rows of one image, or 128 rows where the batch is too small to give
// every resident block several long segments) and walks it top to bottom in
// chunks of 32 rows.
// For every chunk it computes the separable row pass (smoothing, first- and
// second-derivative taps along x) of the 32 new rows into a rolling buffer
// that keeps the 2R rows shared with the previous chunk, so the row pass costs
// 3 (2R+1) FMAs per pixel plus 2R halo rows per segment instead of a full
// halo per tile.  The column pass then runs only at the chunk's pixels whose
// selected scale is this one, and (with the scale image's chunk masks) only on
// the chunks that hold such a pixel, the row pass only on the rows those
// chunks read.  The radius R is a template parameter: every tap
// loop is unrolled and the weights are kernel parameters (constant-bank
// operands of the FMAs).  The arithmetic and summation order are those of the
// multi-scale sweep in fd4_scale.cu (which selects on tile lists), so both give
// identical results.
//
// The same kernels run the selection (a dense column pass and the vesselness
// factors of every pixel at each scale) and the IFOD comparator of Eq. 2 (a
// dense column pass at one scale and the tensor (1, 0, g, g) with
// g = 1 / (1 + |H(u_sigma)|_F^2 / lambda^2)).
#include <cmath>
#include <cstdint>

#include "fd4_internal.h"

namespace fd4 {
namespace {

constexpr int ST_TX = 32;    // strip width
constexpr int ST_CH = 32;    // rows per chunk
constexpr int ST_NT = 256;   // threads: row pass = 32 rows x 8 units of 4 outputs
constexpr int ST_RS = 36;    // row-pass buffer stride (16-byte rows)

template <int R>
struct StripTaps {
    float w0[2 * R + 1], w1[2 * R + 1], w2[2 * R + 1];  // tap i at offset i - R
    // the same taps in pairs (w[i], w[i - 1]), i = 0 .. 2R + 1, zero outside
    // 0 .. 2R: the weights of two adjacent outputs for one input value
    float2 p0[2 * R + 2], p1[2 * R + 2], p2[2 * R + 2];
    // pairs of two fields' taps at one offset: (w1[k], w2[k]) and (w0[k], w1[k])
    float2 q12[2 * R + 1], q01[2 * R + 1];
};

__device__ __forceinline__ int st_mirror(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

__device__ __forceinline__ void st_cp16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void st_cp4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void st_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void st_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void st_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int R>
constexpr int st_sw() { return 36 + 2 * R; }  // staged input row stride: >= 32 + 2R, == 4 mod 8

// NS scales of one padded radius R per launch (the tensor build pairs equal
// radii): NS row-pass buffers of three fields share one staged input.
template <int R, int NS = 1>
constexpr size_t st_smem_bytes()
{
    return sizeof(float) * ((size_t)2 * ST_CH * st_sw<R>() + (size_t)3 * NS * (ST_CH + 2 * R) * ST_RS);
}

// The taps of the NS scales of one launch.
template <int R, int NS>
struct StripTapsN {
    StripTaps<R> t[NS];
};

// A segment is walked as a sequence of pieces, each the row pass of up to
// ST_CH rows into the rolling buffer, listed by a plan (SegGeo::code).  A
// "fill" piece k (k < NP0) of chunk c writes buffer rows 32k .. of the NB = 32 +
// 2R rows chunk c's column pass reads (image rows ys + 32c - R + 32k ..); a
// "roll" piece of chunk c keeps the 2R rows chunk c shares with chunk c - 1
// and adds its 32 new rows (image rows ys + 32c + R ..).  Code byte: bits 0-3
// the chunk, bits 4-6 the fill index k or NP0 for a roll, bit 7 set where the
// chunk's column pass runs after the piece.
template <int R>
struct Piece {
    static constexpr int NB = ST_CH + 2 * R, NP0 = (NB + ST_CH - 1) / ST_CH;
    static_assert(NP0 >= 2 && NP0 < 8, "a fill takes 2 .. 7 pieces");
    int ya, b0, n, chunk;  // first image row, first buffer row, rows, chunk it belongs to
    bool roll;             // shift the shared rows down first
    bool col;              // the chunk's buffer is complete and its column pass runs
    __device__ __forceinline__ Piece(int ys, unsigned code)
    {
        chunk = code & 15u;
        const int k = (code >> 4) & 7u;
        col = (code >> 7) & 1u;
        if (k < NP0) {
            ya = ys + ST_CH * chunk - R + ST_CH * k;
            b0 = ST_CH * k;
            n = min(ST_CH, NB - ST_CH * k);
            roll = false;
        } else {
            ya = ys + ST_CH * chunk + R;
            b0 = 2 * R;
            n = ST_CH;
            roll = true;
        }
    }
};

// cp.async of image rows ya .. ya + n - 1 (mirrored), columns x0 - R .. x0 + 31 + R.
template <int R>
__device__ __forceinline__ void st_stage(float *tin, const float *img, int w, int h, int pitch, int x0, int ya,
                                         int n)
{
    constexpr int SW = st_sw<R>(), NC = 32 + 2 * R;
    const int tid = threadIdx.x;
    if (x0 - R >= 0 && x0 + 32 + R <= w) {  // 16-byte chunks: x0 - R and the pitch are multiples of 4
        for (int i = tid; i < n * (NC / 4); i += ST_NT) {
            const int r = i / (NC / 4), c = (i - r * (NC / 4)) * 4;
            st_cp16(tin + r * SW + c, img + (size_t)st_mirror(ya + r, h) * pitch + x0 - R + c);
        }
    } else {
        for (int i = tid; i < n * NC; i += ST_NT) {
            const int r = i / NC, c = i - r * NC;
            st_cp4(tin + r * SW + c, img + (size_t)st_mirror(ya + r, h) * pitch + st_mirror(x0 - R + c, w));
        }
    }
}

// Row pass of staged rows 0 .. n - 1 into buffer rows b0 .. b0 + n - 1: thread
// (row tid / 8, columns 4 (tid % 8) .. + 3), three fields, in packed pair FMAs
// (two FP32 lanes per instruction): outputs (0, 1) and (2, 3) of a thread form
// pairs that take one input value with the tap pair (w[i], w[i - 1]).  Each
// output receives the products w[i] u[x + i - R] in increasing i (plus exact
// zeros at the ends), the order of the multi-scale sweep in fd4_scale.cu.
template <int R>
__device__ __forceinline__ void st_rows2(const StripTaps<R> &tp, const float *tin, float *trow, int b0, int n)
{
    constexpr int SW = st_sw<R>(), NB = ST_CH + 2 * R;
    const int tid = threadIdx.x;
    const int r = tid >> 3, xo = (tid & 7) * 4;
    if (r < n) {
        const float *src = tin + r * SW + xo;
        float2 a0[2], a1[2], a2[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) a0[j] = a1[j] = a2[j] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m4 = 0; m4 < (2 * R + 4 + 3) / 4; ++m4) {
            const float4 v = *reinterpret_cast<const float4 *>(src + 4 * m4);
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 x2 = make_float2(vv[e], vv[e]);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int i = 4 * m4 + e - 2 * j;  // pair index of outputs 2j, 2j + 1
                    if (i >= 0 && i <= 2 * R + 1) {
                        a0[j] = __ffma2_rn(tp.p0[i], x2, a0[j]);
                        a1[j] = __ffma2_rn(tp.p1[i], x2, a1[j]);
                        a2[j] = __ffma2_rn(tp.p2[i], x2, a2[j]);
                    }
                }
            }
        }
        float *d = trow + (b0 + r) * ST_RS + xo;
        *reinterpret_cast<float4 *>(d) = make_float4(a0[0].x, a0[0].y, a0[1].x, a0[1].y);
        *reinterpret_cast<float4 *>(d + NB * ST_RS) = make_float4(a1[0].x, a1[0].y, a1[1].x, a1[1].y);
        *reinterpret_cast<float4 *>(d + 2 * NB * ST_RS) = make_float4(a2[0].x, a2[0].y, a2[1].x, a2[1].y);
    }
}

// The row pass of st_rows2 with warp w computing columns 4w .. 4w + 3 of every
// row (lane = row), so that a unit no chunk reads (bit w of units clear) is
// skipped by its whole warp.  Each output gets the same operations in the
// same order as in st_rows2.
template <int R>
__device__ __forceinline__ void st_rows_units(const StripTaps<R> &tp, const float *tin, float *trow, int b0, int n,
                                              unsigned units)
{
    constexpr int SW = st_sw<R>(), NB = ST_CH + 2 * R;
    const int r = threadIdx.x & 31, xo = (threadIdx.x >> 5) * 4;
    if (!((units >> (threadIdx.x >> 5)) & 1u) || r >= n) return;
    const float *src = tin + r * SW + xo;
    float2 a0[2], a1[2], a2[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) a0[j] = a1[j] = a2[j] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int m4 = 0; m4 < (2 * R + 4 + 3) / 4; ++m4) {
        const float4 v = *reinterpret_cast<const float4 *>(src + 4 * m4);
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 x2 = make_float2(vv[e], vv[e]);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int i = 4 * m4 + e - 2 * j;
                if (i >= 0 && i <= 2 * R + 1) {
                    a0[j] = __ffma2_rn(tp.p0[i], x2, a0[j]);
                    a1[j] = __ffma2_rn(tp.p1[i], x2, a1[j]);
                    a2[j] = __ffma2_rn(tp.p2[i], x2, a2[j]);
                }
            }
        }
    }
    float *d = trow + (b0 + r) * ST_RS + xo;
    *reinterpret_cast<float4 *>(d) = make_float4(a0[0].x, a0[0].y, a0[1].x, a0[1].y);
    *reinterpret_cast<float4 *>(d + NB * ST_RS) = make_float4(a1[0].x, a1[0].y, a1[1].x, a1[1].y);
    *reinterpret_cast<float4 *>(d + 2 * NB * ST_RS) = make_float4(a2[0].x, a2[0].y, a2[1].x, a2[1].y);
}

// Per-launch scalars of the strip kernels.
struct StripArgs {
    int s;          // scale index in the set
    int K_total;    // size of the set
    int grad_sq;    // tensor build: |grad u|^2 instead of |grad u| in the normalisation
    int mode;       // selection: FD4_RIDGE / FD4_VALLEY / FD4_BOTH
    float scale4;   // selection: sigma^(4 gamma)
    float inv2b2;   // selection: 1 / (2 beta^2)
    int shape;      // SHAPE_SEG or SHAPE_SEG_S
    int seg;        // its rows
    float inv_lam2; // IFOD: 1 / lambda^2
    int soa;        // IFOD: the FED coefficient planes (g, 0, 0) instead of (1, 0, g, g)
};

// What a strip launch computes (the kernels' MODE).
enum StripMode {
    ST_TENSOR = 0,  // N at the pixels whose selected scale this is (sparse column pass)
    ST_SELECT = 1,  // vesselness planes of this scale at every pixel (dense column pass)
    ST_IFOD = 2     // IFOD tensor (1, 0, g, g), g = 1 / (1 + |H|_F^2 / lambda^2), at every pixel
};

// Geometry of one strip segment and the plan of its pieces, computed once by
// the thread that looks the segment up (the other threads read it from shared
// memory, so no thread divides by the image's strip count per piece).
constexpr int kMaxPlan = 24;  // pieces of a 512-row segment: at most NP0 - 1 + 16 <= 19
static_assert(kSegRows / ST_CH <= 16, "chunk index in 4 bits");
struct SegGeo {
    int x0, ys;    // first column and row
    int pieces;    // plan length (0: nothing of this segment is needed)
    unsigned char code[kMaxPlan];
    // per chunk: the 4-column units of the row pass its pieces compute (bit u:
    // columns 4u .. 4u + 3), the units the chunks that read those rows need
    unsigned char uni[kSegRows / ST_CH];
};

// The plan of a segment.  Dense launches (selection, IFOD) and images without
// chunk masks run every chunk: NP0 fill pieces, then one roll per chunk.  The
// tensor build runs the column pass only on the chunks that hold a pixel of
// scale s, and the row pass only for the rows those chunks read: between two
// such chunks the buffer rolls through the chunks in between or is filled
// afresh, whichever passes fewer rows (a segment without such a chunk has an
// empty plan).  Every row the column pass reads is computed as in the dense
// walk, so the sums are unchanged.
template <int R>
__device__ __forceinline__ void seg_geo(const ImgDesc &d, int local, int seg, SegGeo &g)
{
    const int tiles_x = (d.w + ST_TX - 1) / ST_TX;
    const int ty = local / tiles_x;
    g.x0 = (local - ty * tiles_x) * ST_TX;
    g.ys = ty * seg;
}

// The plan from the chunks to visit (bit c of need: chunk c of the segment).
template <int R>
__device__ __forceinline__ int seg_plan(unsigned need, int nch, SegGeo &g)
{
    constexpr int NP0 = Piece<R>::NP0, NB = Piece<R>::NB;
    int np = 0, prev = -1;
    for (int c = 0; c < nch; ++c) {
        if (!((need >> c) & 1u)) continue;
        if (prev >= 0 && (c - prev) * ST_CH <= NB) {
            for (int cc = prev + 1; cc < c; ++cc) g.code[np++] = (unsigned char)(cc | (NP0 << 4));
            g.code[np++] = (unsigned char)(c | (NP0 << 4) | 0x80);
        } else {
            for (int k = 0; k < NP0; ++k) g.code[np++] = (unsigned char)(c | (k << 4) | (k == NP0 - 1 ? 0x80 : 0));
        }
        prev = c;
    }
    return np;
}

// Warp 0: the block's next segment with a non-empty plan, from flat segment t
// on in steps of the grid: its descriptor, index in its image and plan into
// the slot (written by lane 0); the segment's number (>= I.tiles: none left).
// Lane c reads the chunk mask of chunk c, so one segment costs one round trip
// to memory.
template <int R, int NS>
__device__ __forceinline__ int next_segment(const Imgs &I, const StripArgs &sa, bool dense, int t, TileCache &tc,
                                            ImgDesc &d, int &local, SegGeo &g)
{
    const int lane = threadIdx.x & 31;
    for (; t < I.tiles; t += gridDim.x) {
        if (lane == 0) {
            find_tile_cached(I, sa.shape, t, tc, d, local);
            seg_geo<R>(d, local, sa.seg, g);
        }
        __syncwarp();
        const int nch = (min(g.ys + sa.seg, d.h) - g.ys + ST_CH - 1) / ST_CH;
        unsigned need = nch >= 32 ? 0xffffffffu : (1u << nch) - 1u;
        unsigned uu = 0xffu;  // lane c: units of chunk c's pieces
        if (!dense && d.cmask) {
            const int cw = (d.w + 31) / 32;
            bool bit = false;
            unsigned um = 0u;
            if (lane < nch) {
                const size_t ch = (size_t)(g.ys / ST_CH + lane) * cw + g.x0 / ST_TX;
                bit = (d.cmask[ch] >> sa.s) & ((1u << NS) - 1u);
                const uint8_t *up = chunk_units(d) + ch * FD4_MAX_SIGMAS + sa.s;
                for (int k = 0; k < NS; ++k) um |= up[k];
            }
            need = __ballot_sync(0xffffffffu, bit);
            // the rows of chunk c's pieces are read by chunks c .. c + (NB - 1) / 32
            uu = um;
            for (int k = 1; k <= (ST_CH + 2 * R - 1) / ST_CH; ++k) uu |= __shfl_down_sync(0xffffffffu, um, k);
        }
        if (lane < kSegRows / ST_CH) g.uni[lane] = (unsigned char)uu;
        if (lane == 0) g.pieces = seg_plan<R>(need, nch, g);
        __syncwarp();
        if (g.pieces > 0) break;
        __syncwarp();  // every lane has read g before lane 0 rewrites it
    }
    return t;
}

// Scale s (radius R) over every strip segment of the batch, or the NS scales
// s .. s + NS - 1 of one padded radius (tensor build only).
// Tensor build (ST_TENSOR): idx holds each pixel's selected scale; only pixels
// with idx in s .. s + NS - 1 are written (nfield), and the s == 0 launch also
// zeroes N where idx lies outside the scale set.  Selection (ST_SELECT): every pixel's Hessian
// at scale s gives the vesselness factor and S^2 of plane s (vp, s2) and the
// image's max S^2.  The next piece's rows (of this segment or of the block's
// next one) are copied with cp.async while the current piece is computed.
template <int R, int MODE, int NS>
__global__ void __launch_bounds__(ST_NT) k_strip(Imgs I, StripTapsN<R, NS> tpn, StripArgs sa)
{
    constexpr bool SEL = MODE == ST_SELECT, DENSE = MODE != ST_TENSOR;
    // the pair of the smallest radius (its two scales cover most pixels of a
    // noisy image) takes the dense column pass of both scales; at R = 8 and 12
    // the pixel list is faster (measured: 191 / 214 against 251 / 261 us per
    // 4096^2 launch), at R = 4 the dense pass (193 against 228 us)
    constexpr bool PAIR = MODE == ST_TENSOR && NS == 2 && R <= 4;
    static_assert(NS == 1 || !DENSE, "scales share a launch in the tensor build only");
    constexpr int NB = ST_CH + 2 * R, SW = st_sw<R>();
    const StripTaps<R> &tp = tpn.t[0];
    extern __shared__ __align__(16) float stsm[];
    // staged rows: two ST_CH x SW buffers; then per scale 3 fields x NB rows x ST_RS
    float *trow = stsm + 2 * ST_CH * SW;
    constexpr int NL = (DENSE || PAIR) ? 1 : NS;  // pixel lists: the sparse column pass only
    __shared__ unsigned short plist[NL][ST_TX * ST_CH];
    __shared__ int wtot[NL][ST_NT / 32];
    __shared__ ImgDesc sd[2];
    __shared__ int s_local[2];
    __shared__ SegGeo sg[2];
    __shared__ int s_t[2];  // flat segment number of each slot
    __shared__ TileCache tcache;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, s = sa.s;
    float bmax = 0.0f;  // selection: max S^2 of this thread's pixels in the current segment
    if (blockIdx.x >= I.tiles) return;
    if (tid == 0) tc_reset(tcache);
    if (warp == 0) {
        __syncwarp();
        const int tt = next_segment<R, NS>(I, sa, DENSE, blockIdx.x, tcache, sd[0], s_local[0], sg[0]);
        if (lane == 0) s_t[0] = tt;
    }
    __syncthreads();
    int t = s_t[0];
    if (t >= I.tiles) return;  // block-uniform: no segment of this block needs scale s
    int cur = 0, i = 0, buf = 0;
    {
        const Piece<R> p0(sg[0].ys, sg[0].code[0]);
        st_stage<R>(stsm, SEL ? sd[0].in : sd[0].u, sd[0].w, sd[0].h, sd[0].pitch, sg[0].x0, p0.ya, p0.n);
        st_commit();
    }
    for (;;) {
        const int w = sd[cur].w, h = sd[cur].h, pitch = sd[cur].pitch;
        const int x0 = sg[cur].x0, ys = sg[cur].ys, P = sg[cur].pieces;
        const Piece<R> pc(ys, sg[cur].code[i]);
        // issue the next piece into the other staging buffer; the next segment
        // was looked up at piece 0 and published by that piece's barriers (a
        // non-empty plan has at least NP0 >= 2 pieces)
        float *nbuf = stsm + (buf ^ 1) * ST_CH * SW;
        if (i + 1 < P) {
            const Piece<R> pn(ys, sg[cur].code[i + 1]);
            st_stage<R>(nbuf, SEL ? sd[cur].in : sd[cur].u, w, h, pitch, x0, pn.ya, pn.n);
        } else if (s_t[cur ^ 1] < I.tiles) {
            const ImgDesc &dn = sd[cur ^ 1];
            const Piece<R> pn(sg[cur ^ 1].ys, sg[cur ^ 1].code[0]);
            st_stage<R>(nbuf, SEL ? dn.in : dn.u, dn.w, dn.h, dn.pitch, sg[cur ^ 1].x0, pn.ya, pn.n);
        }
        st_commit();
        // the selected scales of the chunk this piece completes (rows 4 warp .. + 3)
        const int y0 = ys + ST_CH * pc.chunk;
        int ids[4] = {-1, -1, -1, -1};
        if (!DENSE && pc.col && x0 + lane < w) {
            const uint8_t *ip = sd[cur].idx + (size_t)(y0 + warp * 4) * pitch + x0 + lane;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (y0 + warp * 4 + j < h) ids[j] = ip[(size_t)j * pitch];
        }
        st_wait1();
        __syncthreads();  // this piece's rows have landed; the previous chunk's column pass is done
        // the block's next segment: its slot held the previous segment, whose last
        // readers (the column pass above) are past this barrier
        if (i == 0 && warp == 0) {
            const int tt =
                next_segment<R, NS>(I, sa, DENSE, t + G, tcache, sd[cur ^ 1], s_local[cur ^ 1], sg[cur ^ 1]);
            if (lane == 0) s_t[cur ^ 1] = tt;
        }
        if (pc.roll) {
            // keep buffer rows ST_CH .. ST_CH + 2R - 1 as rows 0 .. 2R - 1.
            // Thread (row r, columns c .. c + 3) moves rows k0 + r for k0 = 0,
            // 32, ...: a row it overwrites in pass k0 + 32 is one it read
            // itself in pass k0, so the passes need no barrier between them.
            const int r = tid >> 3, c = (tid & 7) * 4;
#pragma unroll
            for (int k0 = 0; k0 < 2 * R; k0 += ST_CH) {
                if (k0 + r < 2 * R) {
#pragma unroll
                    for (int f = 0; f < 3 * NS; ++f) {
                        float *fb = trow + f * NB * ST_RS;
                        *reinterpret_cast<float4 *>(fb + (k0 + r) * ST_RS + c) =
                            *reinterpret_cast<const float4 *>(fb + (ST_CH + k0 + r) * ST_RS + c);
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int ns = 0; ns < NS; ++ns) {
            // single-scale launches (R >= 16 here) compute only the units their
            // chunks read (the pairs' units are nearly all read: the row-per-thread
            // mapping measured faster there)
            if constexpr (!DENSE && !PAIR && NS == 1)
                st_rows_units<R>(tpn.t[ns], stsm + buf * ST_CH * SW, trow + ns * 3 * NB * ST_RS, pc.b0, pc.n,
                                 sg[cur].uni[pc.chunk]);
            else
                st_rows2<R>(tpn.t[ns], stsm + buf * ST_CH * SW, trow + ns * 3 * NB * ST_RS, pc.b0, pc.n);
        }
        __syncthreads();

        if (DENSE && pc.col) {
            // dense column pass: column lane, rows 4 warp .. + 3 of the chunk
            // read buffer rows 4 warp .. 4 warp + 3 + 2R
            const float *c0 = trow + (warp * 4) * ST_RS + lane;
            const float *c1 = c0 + NB * ST_RS, *c2 = c1 + NB * ST_RS;
            float uxx[4], uxy[4], uyy[4];
            // output rows (0, 1) and (2, 3) in packed pairs, as in st_rows2
            float2 axx[2], axy[2], ayy[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) axx[j] = axy[j] = ayy[j] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 2 * R + 4; ++k) {
                const float v0 = c0[k * ST_RS], v1 = c1[k * ST_RS], v2 = c2[k * ST_RS];
                const float2 x0 = make_float2(v0, v0), x1 = make_float2(v1, v1), x2 = make_float2(v2, v2);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int q = k - 2 * j;  // tap pair of output rows 2j, 2j + 1
                    if (q >= 0 && q <= 2 * R + 1) {
                        axx[j] = __ffma2_rn(tp.p0[q], x2, axx[j]);
                        axy[j] = __ffma2_rn(tp.p1[q], x1, axy[j]);
                        ayy[j] = __ffma2_rn(tp.p2[q], x0, ayy[j]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uxx[2 * j] = axx[j].x; uxx[2 * j + 1] = axx[j].y;
                uxy[2 * j] = axy[j].x; uxy[2 * j + 1] = axy[j].y;
                uyy[2 * j] = ayy[j].x; uyy[2 * j + 1] = ayy[j].y;
            }
            const int gx = x0 + lane;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gy = y0 + warp * 4 + j;
                if (gx >= w || gy >= h) continue;
                const float a = uxx[j], b = uxy[j], d = uyy[j];
                if (!SEL) {  // IFOD: D = g I
                    const float f2 = fmaf(a, a, fmaf(2.0f * b, b, d * d));
                    const float g = 1.0f / fmaf(f2, sa.inv_lam2, 1.0f);
                    if (sa.soa) {
                        float *tp = reinterpret_cast<float *>(sd[cur].tensor) + (size_t)gy * pitch + gx;
                        const size_t P = fed_coef_plane(h, pitch);
                        tp[0] = g;  // mu3 = (g + g) / 2; q = 0
                        tp[P] = 0.0f;
                        tp[2 * P] = 0.0f;
                    } else {
                        sd[cur].tensor[(size_t)gy * pitch + gx] = make_float4(1.0f, 0.0f, g, g);
                    }
                    continue;
                }
                // eigenvalues of H (sigma^(2 gamma) cancels in R_B and the sign
                // test; S^2 picks it up as sigma^(4 gamma))
                const float m = 0.5f * (a + d);
                const float rr = hypotf(0.5f * (a - d), b);
                const float far = m > 0.0f ? m + rr : m - rr;  // larger magnitude; ties -> negative
                float vp = 0.0f;
                const bool wrong = (sa.mode == FD4_RIDGE && far > 0.0f) || (sa.mode == FD4_VALLEY && far < 0.0f);
                if (!wrong && far != 0.0f) {
                    const float near = det2_sym(a, b, d) / far;  // cancellation-free
                    const float rb = near / far;
                    vp = expf(-rb * rb * sa.inv2b2);
                }
                const float s2 = sa.scale4 * fmaf(a, a, fmaf(2.0f * b, b, d * d));
                const size_t p = (size_t)gy * pitch + gx;
                sd[cur].vp[(size_t)s * sd[cur].plane + p] = vp;
                sd[cur].s2[(size_t)s * sd[cur].plane + p] = s2;
                bmax = fmaxf(bmax, s2);
            }
            if (SEL && i + 1 == P) {  // segment done: fold its max S^2 into the image's
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
                if (lane == 0 && bmax > 0.0f) atomicMax(sd[cur].max_s2, __float_as_uint(bmax));
                bmax = 0.0f;
            }
        }
        if (PAIR && pc.col) {
            // dense column pass of both scales of the pair: column lane, rows
            // 4 warp .. + 3, in packed
            // pairs of output rows as the selection's dense pass; each output gets
            // the products in increasing tap order, as the pixel-list pass below
            float n5[4][5];  // (sx, sy, sxx, sxy, syy) at the pixel's own scale
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (s == 0 && ids[j] >= sa.K_total)
                    sd[cur].nfield[(size_t)(y0 + warp * 4 + j) * pitch + x0 + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int f = 0; f < 5; ++f) n5[j][f] = 0.0f;
            }
#pragma unroll
            for (int ns = 0; ns < NS; ++ns) {
                bool mine = false;
#pragma unroll
                for (int j = 0; j < 4; ++j) mine |= ids[j] == s + ns;
                if (!__any_sync(0xffffffffu, mine)) continue;  // warp-uniform
                const StripTaps<R> &tq = tpn.t[ns];
                const float *c0 = trow + ns * 3 * NB * ST_RS + (warp * 4) * ST_RS + lane;  // smoothed along x
                const float *c1 = c0 + NB * ST_RS;                                         // d/dx
                const float *c2 = c1 + NB * ST_RS;                                         // d2/dx2
                float2 ay[2], ayy[2], ax[2], axy[2], axx[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) ay[j] = ayy[j] = ax[j] = axy[j] = axx[j] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int k = 0; k < 2 * R + 4; ++k) {
                    const float v0 = c0[k * ST_RS], v1 = c1[k * ST_RS], v2 = c2[k * ST_RS];
                    const float2 x0v = make_float2(v0, v0), x1v = make_float2(v1, v1), x2v = make_float2(v2, v2);
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int q = k - 2 * j;  // tap pair of output rows 2j, 2j + 1
                        if (q >= 0 && q <= 2 * R + 1) {
                            ay[j] = __ffma2_rn(tq.p1[q], x0v, ay[j]);
                            ayy[j] = __ffma2_rn(tq.p2[q], x0v, ayy[j]);
                            ax[j] = __ffma2_rn(tq.p0[q], x1v, ax[j]);
                            axy[j] = __ffma2_rn(tq.p1[q], x1v, axy[j]);
                            axx[j] = __ffma2_rn(tq.p0[q], x2v, axx[j]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (ids[j] != s + ns) continue;
                    const int jp = j >> 1;
                    const bool hi = j & 1;
                    n5[j][0] = hi ? ax[jp].y : ax[jp].x;
                    n5[j][1] = hi ? ay[jp].y : ay[jp].x;
                    n5[j][2] = hi ? axx[jp].y : axx[jp].x;
                    n5[j][3] = hi ? axy[jp].y : axy[jp].x;
                    n5[j][4] = hi ? ayy[jp].y : ayy[jp].x;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ids[j] < s || ids[j] >= s + NS) continue;  // (ids is -1 outside the image)
                const float sx = n5[j][0], sy = n5[j][1];
                const float g2 = fmaf(sx, sx, sy * sy);
                const float g = sa.grad_sq ? g2 : sqrtf(g2);
                const float f = 1.0f / sqrtf(1.0f + g);
                sd[cur].nfield[(size_t)(y0 + warp * 4 + j) * pitch + x0 + lane] =
                    make_float4(f * n5[j][2], f * n5[j][3], f * n5[j][4], 0.0f);
            }
        }
        if constexpr (!DENSE && !PAIR) if (pc.col) {
            // the chunk's pixels of each scale, grouped in plist[ns]
            unsigned m[NS][4];
            int cnt[NS];
#pragma unroll
            for (int ns = 0; ns < NS; ++ns) cnt[ns] = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (s == 0 && ids[j] >= sa.K_total)
                    sd[cur].nfield[(size_t)(y0 + warp * 4 + j) * pitch + x0 + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int ns = 0; ns < NS; ++ns) {
                    m[ns][j] = __ballot_sync(0xffffffffu, ids[j] == s + ns);
                    cnt[ns] += __popc(m[ns][j]);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int ns = 0; ns < NS; ++ns) wtot[ns][warp] = cnt[ns];
            }
            __syncthreads();
            int total[NS];
#pragma unroll
            for (int ns = 0; ns < NS; ++ns) {
                // every warp sums the counts itself: its first list slot and the total
                int first;
                {
                    const int c = lane < warp ? wtot[ns][lane] : 0, a = lane < ST_NT / 32 ? wtot[ns][lane] : 0;
                    first = c;
                    total[ns] = a;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {  // every lane ends with the sums
                        first += __shfl_xor_sync(0xffffffffu, first, o);
                        total[ns] += __shfl_xor_sync(0xffffffffu, total[ns], o);
                    }
                }
                int pos = first;
                const unsigned lt = (1u << lane) - 1u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((m[ns][j] >> lane) & 1u)
                        plist[ns][pos + __popc(m[ns][j] & lt)] = (unsigned short)(((warp * 4 + j) << 5) | lane);
                    pos += __popc(m[ns][j]);
                }
            }
            __syncthreads();
            // column pass: output row y0 + py reads buffer rows py .. py + 2R
#pragma unroll
            for (int ns = 0; ns < NS; ++ns) {
                const StripTaps<R> &tq = tpn.t[ns];
                const float *tr = trow + ns * 3 * NB * ST_RS;
                for (int e = tid; e < total[ns]; e += ST_NT) {
                    const int entry = plist[ns][e];
                    const int px = entry & 31, py = entry >> 5;
                    const float *c0 = tr + py * ST_RS + px;   // smoothed along x
                    const float *c1 = c0 + NB * ST_RS;         // d/dx
                    const float *c2 = c1 + NB * ST_RS;         // d2/dx2
                    float sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
                    {  // (sy, syy) and (sx, sxy) share their input: packed pairs
                        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k <= 2 * R; ++k) {
                            const float v0 = c0[k * ST_RS], v1 = c1[k * ST_RS], v2 = c2[k * ST_RS];
                            a = __ffma2_rn(tq.q12[k], make_float2(v0, v0), a);
                            b = __ffma2_rn(tq.q01[k], make_float2(v1, v1), b);
                            sxx = fmaf(tq.w0[k], v2, sxx);
                        }
                        sy = a.x; syy = a.y; sx = b.x; sxy = b.y;
                    }
                    const float g2 = fmaf(sx, sx, sy * sy);
                    const float g = sa.grad_sq ? g2 : sqrtf(g2);
                    const float f = 1.0f / sqrtf(1.0f + g);
                    sd[cur].nfield[(size_t)(y0 + py) * pitch + x0 + px] = make_float4(f * sxx, f * sxy, f * syy, 0.0f);
                }
            }
        }
        buf ^= 1;
        if (++i == P) {
            i = 0;
            t = s_t[cur ^ 1];
            cur ^= 1;
            if (t >= I.tiles) break;
        }
    }
    st_wait0();
}

// Chunk masks of the scale image for the tensor build: for each 32 x 32 chunk,
// bit s set where one of its pixels selected scale s; an index outside the set
// sets bit 0 (the scale-0 launch zeroes N there).  Then per chunk and scale
// the unit mask: bit u set where columns 4u .. 4u + 3 hold a pixel of the
// scale (the strips compute the row pass only for the units some chunk reads).
// 32 x 64 tiles (two chunks), 256 threads: lane = column, warp w = rows
// 8w .. 8w + 7 of the tile.
__global__ void __launch_bounds__(256) k_chunk_masks(Imgs I, int K)
{
    __shared__ ImgDesc sd;
    __shared__ int s_local;
    __shared__ unsigned sm[2];
    __shared__ unsigned su[2][8];  // per chunk and 4-column unit: the scales it holds
    __shared__ TileCache tcache;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tc_reset(tcache);
    for (int t = blockIdx.x; t < I.tiles; t += gridDim.x) {
        __syncthreads();
        if (tid == 0) {
            find_tile_cached(I, SHAPE_SWEEP, t, tcache, sd, s_local);
            sm[0] = sm[1] = 0u;
        }
        if (tid < 16) su[tid >> 3][tid & 7] = 0u;
        __syncthreads();
        const int w = sd.w, h = sd.h, pitch = sd.pitch;
        const int cw = (w + 31) / 32;
        const int x0 = (s_local % cw) * 32, y0 = (s_local / cw) * 64;
        const int x = x0 + lane;
        unsigned m = 0u, mk = 0u;  // all indices; the valid ones (for the unit masks)
        if (x < w) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int y = y0 + warp * 8 + j;
                if (y < h) {
                    const int v = sd.idx[(size_t)y * pitch + x];
                    m |= v < K ? 1u << v : 1u;
                    if (v < K) mk |= 1u << v;
                }
            }
        }
        const unsigned wm = __reduce_or_sync(0xffffffffu, m);
        if (lane == 0) atomicOr(&sm[warp >> 2], wm);
        // the scales of each 4-column unit (lanes 4u .. 4u + 3)
        mk |= __shfl_xor_sync(0xffffffffu, mk, 1);
        mk |= __shfl_xor_sync(0xffffffffu, mk, 2);
        if ((lane & 3) == 0 && mk) atomicOr(&su[warp >> 2][lane >> 2], mk);
        __syncthreads();
        if (tid < 2 && y0 + 32 * tid < h) sd.cmask[(size_t)(y0 / 32 + tid) * cw + x0 / 32] = sm[tid];
        if (tid < 2 * K) {  // unit mask of scale sc: bit u where unit u holds it
            const int c = tid / K, sc = tid - (tid / K) * K;
            unsigned u8 = 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) u8 |= ((su[c][u] >> sc) & 1u) << u;
            if (y0 + 32 * c < h)
                chunk_units(sd)[((size_t)(y0 / 32 + c) * cw + x0 / 32) * FD4_MAX_SIGMAS + sc] = (uint8_t)u8;
        }
    }
}

template <int R, int MODE, int NS>
int launch_strip_k(const Imgs &I, const StripTapsN<R, NS> &tp, const StripArgs &a, cudaStream_t st)
{
    static int attr_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    constexpr size_t smem = st_smem_bytes<R, NS>();
    if (attr_dev != dev) {
        if (cudaFuncSetAttribute(k_strip<R, MODE, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 1;
        attr_dev = dev;
    }
    const int grid = persistent_grid((const void *)k_strip<R, MODE, NS>, ST_NT, smem, I.tiles);
    k_strip<R, MODE, NS><<<grid, ST_NT, smem, st>>>(I, tp, a);
    return cudaGetLastError() != cudaSuccess;
}

// The taps of one scale in the strip kernels' layout (radius R >= g.r).
template <int R>
void strip_taps(const GaussTaps &g, StripTaps<R> &tp)
{
    const float *src[3] = {g.w0, g.w1, g.w2};
    float *dst[3] = {tp.w0, tp.w1, tp.w2};
    float2 *pd[3] = {tp.p0, tp.p1, tp.p2};
    for (int k = 0; k < 3; ++k) {
        for (int i = 0; i <= 2 * R; ++i) {
            const int o = i - R;
            dst[k][i] = (o >= -g.r && o <= g.r) ? src[k][o + g.r] : 0.0f;
        }
        for (int i = 0; i <= 2 * R + 1; ++i)
            pd[k][i] = make_float2(i <= 2 * R ? dst[k][i] : 0.0f, i >= 1 ? dst[k][i - 1] : 0.0f);
    }
    for (int i = 0; i <= 2 * R; ++i) {
        tp.q12[i] = make_float2(tp.w1[i], tp.w2[i]);
        tp.q01[i] = make_float2(tp.w0[i], tp.w1[i]);
    }
}

// NS scales of padded radius R (taps g[0 .. NS-1]) in one launch.
template <int R, int MODE, int NS>
int launch_strip_scale(const HostBatch &B, const GaussTaps *g, const StripArgs &sa, cudaStream_t st)
{
    constexpr size_t smem = st_smem_bytes<R, NS>();
    StripTapsN<R, NS> tp;
    for (int k = 0; k < NS; ++k) strip_taps<R>(g[k], tp.t[k]);
    // Segment length: the one with the smaller estimated time, taken as the
    // rounds of the persistent grid times the rows a block passes per segment
    // (its rows, the 2R halo rows and one chunk for the segment's start, whose
    // staging is not overlapped).
    const int cap = persistent_grid((const void *)k_strip<R, MODE, NS>, ST_NT, smem, 1 << 30);
    const long long rounds_l = (B.tiles[SHAPE_SEG] + cap - 1) / cap;
    const long long rounds_s = (B.tiles[SHAPE_SEG_S] + cap - 1) / cap;
    const bool lng = rounds_l * (kSegRows + 2 * R + ST_CH) <= rounds_s * (kSegRowsShort + 2 * R + ST_CH);
    StripArgs a = sa;
    a.shape = lng ? SHAPE_SEG : SHAPE_SEG_S;
    a.seg = lng ? kSegRows : kSegRowsShort;
    Imgs I = B.I;
    I.tiles = B.tiles[a.shape];
    return launch_strip_k<R, MODE, NS>(I, tp, a, st);
}

// Scales s, s + 1 of one padded radius share a launch in the tensor build
// (one staging and one barrier sequence for both) up to this radius.
constexpr int kMaxPairRadius = 16;

template <int MODE>
int launch_strips(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p, cudaStream_t st)
{
    if (B.I.list) return 1;  // the strips walk whole images, never a tile subset
    for (int s = 0; s < n_sigma;) {
        GaussTaps g[2];
        if (gauss_taps(h_sigmas[s], &g[0]) != FD4_OK) return 1;
        const int R = (g[0].r + 3) / 4 * 4;
        int ns = 1;
        if (MODE == ST_TENSOR && s + 1 < n_sigma && R <= kMaxPairRadius) {
            if (gauss_taps(h_sigmas[s + 1], &g[1]) != FD4_OK) return 1;
            if ((g[1].r + 3) / 4 * 4 == R) ns = 2;
        }
        StripArgs sa;
        sa.s = s;
        sa.K_total = n_sigma;
        sa.grad_sq = p.grad_norm_squared;
        sa.mode = p.mode;
        sa.scale4 = (float)pow((double)h_sigmas[s], 4.0 * p.gamma);
        sa.inv2b2 = (float)(1.0 / (2.0 * (double)p.beta * p.beta));
        sa.inv_lam2 = (float)(1.0 / ((double)p.lambda * p.lambda));
        sa.soa = B.fed_soa ? 1 : 0;
        int rc = 1;
        if constexpr (MODE == ST_TENSOR) {
            if (ns == 2) {
                switch (R) {
                case 4: rc = launch_strip_scale<4, MODE, 2>(B, g, sa, st); break;
                case 8: rc = launch_strip_scale<8, MODE, 2>(B, g, sa, st); break;
                case 12: rc = launch_strip_scale<12, MODE, 2>(B, g, sa, st); break;
                case 16: rc = launch_strip_scale<16, MODE, 2>(B, g, sa, st); break;
                default: rc = 1;
                }
            }
        }
        if (ns == 1) {
            switch (R) {
            case 4: rc = launch_strip_scale<4, MODE, 1>(B, g, sa, st); break;
            case 8: rc = launch_strip_scale<8, MODE, 1>(B, g, sa, st); break;
            case 12: rc = launch_strip_scale<12, MODE, 1>(B, g, sa, st); break;
            case 16: rc = launch_strip_scale<16, MODE, 1>(B, g, sa, st); break;
            case 20: rc = launch_strip_scale<20, MODE, 1>(B, g, sa, st); break;
            case 24: rc = launch_strip_scale<24, MODE, 1>(B, g, sa, st); break;
            case 28: rc = launch_strip_scale<28, MODE, 1>(B, g, sa, st); break;
            case 32: rc = launch_strip_scale<32, MODE, 1>(B, g, sa, st); break;
            case 36: rc = launch_strip_scale<36, MODE, 1>(B, g, sa, st); break;
            case 40: rc = launch_strip_scale<40, MODE, 1>(B, g, sa, st); break;
            case 44: rc = launch_strip_scale<44, MODE, 1>(B, g, sa, st); break;
            case 48: rc = launch_strip_scale<48, MODE, 1>(B, g, sa, st); break;
            default: rc = 1;
            }
        }
        if (rc) return 1;
        s += ns;
    }
    return 0;
}

template <int R>
int set_strip_smem()
{
    const int b = (int)st_smem_bytes<R>();
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if constexpr (R <= kMaxPairRadius) {
        if (cudaFuncSetAttribute(k_strip<R, ST_TENSOR, 2>, a, (int)st_smem_bytes<R, 2>()) != cudaSuccess) return 1;
    }
    return cudaFuncSetAttribute(k_strip<R, ST_TENSOR, 1>, a, b) != cudaSuccess ||
           cudaFuncSetAttribute(k_strip<R, ST_SELECT, 1>, a, b) != cudaSuccess ||
           cudaFuncSetAttribute(k_strip<R, ST_IFOD, 1>, a, b) != cudaSuccess;
}

}  // namespace

int prepare_tensor_kernels()
{
    return set_strip_smem<4>() || set_strip_smem<8>() || set_strip_smem<12>() || set_strip_smem<16>() ||
           set_strip_smem<20>() || set_strip_smem<24>() || set_strip_smem<28>() || set_strip_smem<32>() ||
           set_strip_smem<36>() || set_strip_smem<40>() || set_strip_smem<44>() || set_strip_smem<48>();
}

// N at each pixel's selected scale for every image of the batch (nfield).
int launch_tensor_strips(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                         cudaStream_t st)
{
    if (B.has_cmask && !B.cmask_fresh) {  // which chunks hold which scales: the strips skip the others
        Imgs I = B.I;
        I.tiles = B.tiles[SHAPE_SWEEP];
        const int grid = persistent_grid((const void *)k_chunk_masks, 256, 0, I.tiles);
        k_chunk_masks<<<grid, 256, 0, st>>>(I, n_sigma);
        if (cudaGetLastError() != cudaSuccess) return 1;
    }
    return launch_strips<ST_TENSOR>(B, h_sigmas, n_sigma, p, st);
}

// Selection planes (vp, s2) of every scale and each image's max S^2 (which the
// caller clears first).
int launch_select_strips(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                         cudaStream_t st)
{
    return launch_strips<ST_SELECT>(B, h_sigmas, n_sigma, p, st);
}

// IFOD tensor field (1, 0, g, g) of every image of the batch from u: one dense
// strip launch at the regularisation scale sigma.
int launch_ifod_tensor(const HostBatch &B, float sigma, const fd4_params &p, cudaStream_t st)
{
    return launch_strips<ST_IFOD>(B, &sigma, 1, p, st);
}

}  // namespace fd4
