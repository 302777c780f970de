// Internal declarations shared by the fd4 translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fd4.h"

namespace fd4 {

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
// (null if the driver does not provide it).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();

constexpr int kMaxRadius = 48;              // ceil(4 * FD4_MAX_SIGMA)
constexpr int kMaxTaps = 2 * kMaxRadius + 1;
constexpr int kMaxRhoRadius = 8;            // G_rho radius limit (rho <= 2)
constexpr size_t kHeaderBytes = 256;        // status word, max S^2, spare

// Correlation weights of one Gaussian scale: out[x] = sum_k w[k + r] in[x + k].
// w0 smooths, w1 is the first derivative, w2 the second (Sec. 3.1, Eq. 6).
struct GaussTaps {
    int r;
    float w0[kMaxTaps];
    float w1[kMaxTaps];
    float w2[kMaxTaps];
};

struct RhoTaps {
    int r;
    float w0[2 * kMaxRhoRadius + 1];
};

// Device-side header at the start of every workspace.
struct WsHeader {
    int status;          // FD4_OK or a device-detected fd4_status
    unsigned max_s2;     // max of S^2 as float bits (non-negative floats order as ints)
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// Batches.  Every stage kernel walks a flat list of tiles that spans all images
// of a batch (a persistent grid striding over the list); the tile shape
// depends on the kernel.
// SHAPE_SEG / SHAPE_SEG_S: a 32-column strip segment of 512 / 128 rows (the
// strip kernels walk it top to bottom; the short form for batches too small
// to fill the GPU with long segments).
enum TileShape {
    SHAPE_SWEEP = 0,
    SHAPE_SMALL = 1,
    SHAPE_FUSE2 = 2,   // 64 x 32 regions, (64 - 4S) x (32 - 4S) outputs, S = 2 (also the TMA kernel's 32-row form)
    SHAPE_FUSE3 = 3,   //   ... S = 3
    SHAPE_FUSE4 = 4,   //   ... S = 4
    SHAPE_SEG = 5,
    SHAPE_Q64_2 = 6,   // quad FED kernel on 64 x 64 regions: (64 - 4S)^2 outputs, S = 2
    SHAPE_Q64_4 = 7,   //   ... S = 4
    SHAPE_SEG_S = 8,
    kShapes = 9
};
constexpr int kSegRows = 512, kSegRowsShort = 128;

__host__ __device__ inline int shape_tx(int s)
{
    if (s == SHAPE_SWEEP || s == SHAPE_SMALL || s == SHAPE_SEG || s == SHAPE_SEG_S) return 32;
    if (s == SHAPE_Q64_2) return 56;
    if (s == SHAPE_Q64_4) return 48;
    return 64 - 4 * s;
}
__host__ __device__ inline int shape_ty(int s)
{
    if (s == SHAPE_SWEEP) return 64;
    if (s == SHAPE_SMALL) return 8;
    if (s == SHAPE_SEG) return kSegRows;
    if (s == SHAPE_SEG_S) return kSegRowsShort;
    if (s == SHAPE_Q64_2) return 56;
    if (s == SHAPE_Q64_4) return 48;
    return 32 - 4 * s;
}

// Per-image pointers and sizes of one batch entry (planes laid out by the host).
struct ImgDesc {
    const float *in;     // image read by scale selection
    float *u;            // image filtered in place (tensor build input, FED state)
    float *tmp;          // FED ping-pong plane
    float *vp, *s2;      // selection planes, n_sigma each, `plane` floats apart
    float4 *nfield;      // normalised Hessian (Nxx, Nxy, Nyy, 0)
    float4 *tensor;      // (cos 2t, sin 2t, mu1, mu2)
    uint8_t *idx;        // selected scale index
    uint8_t *idx2;       // post-processed scale index before its copy into idx
    float *vmax;         // nullable (set when the scale image is post-processed)
    uint32_t *cmask;     // nullable: per 32 x 32 chunk of the scale image, bit s set where a
                         // pixel selected scale s (an index outside the set counts as 0); then
                         // per chunk 32 unit masks (chunk_units)
    unsigned *max_s2;    // max S^2 of the image (float bits)
    size_t plane;
    const void *maps;    // batches: this image's TMA tensor maps (u, FED plane, tensor) in device memory
    int w, h, pitch;
    int t0[kShapes];     // first flat tile of this image, per tile shape
};

// A batch: a device table of n descriptors, or (table == nullptr) one inline.
struct Imgs {
    const ImgDesc *table;
    int n;
    int tiles;           // total tiles for the launched kernel's shape
    ImgDesc one;
    // Optional subset (single image, sweep tiles): list[0 .. *count) holds the
    // SHAPE_SWEEP tiles to process; a SHAPE_SMALL kernel then processes the 8
    // small tiles (32 x 8) covering each listed 32 x 64 sweep tile.
    const int *list;
    const int *count;
};

inline int tiles_of(int w, int h, int shape)
{
    return ((w + shape_tx(shape) - 1) / shape_tx(shape)) * ((h + shape_ty(shape) - 1) / shape_ty(shape));
}

// Fills d.t0 for a single image and returns the inline batch for `shape`.
inline Imgs single(const ImgDesc &d0, int shape)
{
    Imgs I;
    I.table = nullptr;
    I.list = nullptr;
    I.count = nullptr;
    I.n = 1;
    I.one = d0;
    for (int s = 0; s < kShapes; ++s) I.one.t0[s] = 0;
    I.tiles = tiles_of(d0.w, d0.h, shape);
    return I;
}

#ifdef __CUDACC__
// Thread 0 of a block: the descriptor of flat tile t (shape `shape`) and the
// tile's index within its image.
__device__ __forceinline__ void find_tile(const Imgs &I, int shape, int t, ImgDesc &out, int &local)
{
    if (I.table == nullptr) {
        out = I.one;
        local = t;
        if (I.list) {
            if (shape == SHAPE_SWEEP) {
                local = I.list[t];
            } else {  // small tile k of listed sweep tile t / 8 (both tile grids are 32 wide)
                const int st = I.list[t >> 3], tx = (out.w + 31) / 32;
                local = (8 * (st / tx) + (t & 7)) * tx + st % tx;
            }
        }
        return;
    }
    int lo = 0, hi = I.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (I.table[mid].t0[shape] <= t) lo = mid;
        else hi = mid - 1;
    }
    out = I.table[lo];
    local = t - out.t0[shape];
}
// a d - b^2 with Kahan's fma compensation (error analysed by Jeannerod,
// Louvet and Muller, Math. Comp. 2013): accurate even under cancellation.
__device__ __forceinline__ float det2_sym(float a, float b, float d)
{
    const float bb = b * b;
    const float err = fmaf(-b, b, bb);
    return fmaf(a, d, -bb) + err;
}

// Per-block cache of the last image find_tile_cached resolved: its tile range
// [lo, hi) for one tile shape and its descriptor.  Kept in shared memory;
// tc_reset empties it.
struct TileCache {
    int lo, hi;
    ImgDesc d;
};
__device__ __forceinline__ void tc_reset(TileCache &c)
{
    c.lo = 1;
    c.hi = 0;
}

// Thread 0 of a block: as find_tile, but a persistent block's tiles (t, t +
// gridDim.x, ...) advance through the batch in image order, so most look-ups
// stay within the cached image and need no search of the descriptor table in
// global memory (each step of which is a dependent load).
__device__ __forceinline__ void find_tile_cached(const Imgs &I, int shape, int t, TileCache &c, ImgDesc &out,
                                                 int &local)
{
    if (I.table == nullptr || I.list) {
        find_tile(I, shape, t, out, local);
        return;
    }
    if (t < c.lo || t >= c.hi) {
        int lo = 0, hi = I.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (I.table[mid].t0[shape] <= t) lo = mid;
            else hi = mid - 1;
        }
        c.d = I.table[lo];
        c.lo = c.d.t0[shape];
        c.hi = lo + 1 < I.n ? I.table[lo + 1].t0[shape] : 0x7fffffff;
    }
    out = c.d;
    local = t - c.lo;
}

// Number of tiles a persistent kernel walks: the host count, or the device
// count of a tile list (8 small tiles per listed sweep tile).
__device__ __forceinline__ int tile_count(const Imgs &I, int shape)
{
    if (I.list) return shape == SHAPE_SWEEP ? *I.count : 8 * *I.count;
    return I.tiles;
}
#endif

// Persistent grid size for a kernel: resident blocks per SM x SMs, capped by the tiles.
int persistent_grid(const void *kernel, int threads, size_t smem, int tiles);
// Divides every following persistent grid (used while two streams share the GPU).
void set_grid_divisor(int d);

// Host helpers (fd4_host.cpp).
int gauss_taps(double sigma, GaussTaps *out);            // radius ceil(4 sigma)
int rho_taps(double rho, RhoTaps *out);
int check_image(const void *d, int w, int h, int pitch);
int check_sigmas(const float *h_sigmas, int n_sigma);
void resolve_params(const fd4_params *in, fd4_params *out);
size_t plane_bytes(int h, int pitch, size_t elem);

// Workspace layouts.
size_t ws_select_bytes(int h, int pitch, int n_sigma);
size_t ws_tensor_bytes(int h, int pitch);
size_t ws_fed_bytes(int h, int pitch);
size_t ws_filter_bytes(int h, int pitch, int n_sigma);

// Host view of a batch: the device-visible batch, the total tile count per
// tile shape, and the images' max-S^2 words (contiguous) cleared before selection.
struct HostBatch {
    Imgs I;
    int tiles[kShapes];
    unsigned *max_s2;
    int n_max_s2;
    const ImgDesc *table_u;  // batches: the descriptor table with in = u (nullptr for single images)
    const ImgDesc *table_sw; // batches: the descriptor table with u and the FED plane exchanged
                             // (their TMA maps too); nullptr where the two cannot trade roles
    bool has_cmask;          // every descriptor has its chunk-mask plane (cmask)
    bool cmask_fresh;        // the chunk masks already describe the current scale image
    bool fed_soa;            // ImgDesc::tensor holds the FED coefficient planes (fed_coef_plane)
                             // instead of float4 (cos 2t, sin 2t, mu1, mu2) per pixel
};

// The FED coefficient planes of an image's tensor plane (16 B per pixel): three
// float planes of h x pitch, mu3 = (mu1 + mu2) / 2, q cos 2t and q sin 2t with
// q = (mu1 - mu2) / 4 -- what the TMA FED kernel reads (12 B per pixel).  A
// filter builds them when its FED schedule runs that kernel.
__host__ __device__ inline size_t fed_coef_plane(int h, int pitch) { return (size_t)h * pitch; }

// One image: inline descriptor.
inline HostBatch single_batch(const ImgDesc &d)
{
    HostBatch B;
    B.I = single(d, SHAPE_SWEEP);
    for (int s = 0; s < kShapes; ++s) B.tiles[s] = tiles_of(d.w, d.h, s);
    B.max_s2 = d.max_s2;
    B.n_max_s2 = 1;
    B.table_u = nullptr;
    B.table_sw = nullptr;
    B.has_cmask = d.cmask != nullptr;
    B.cmask_fresh = false;
    B.fed_soa = false;
    return B;
}

// Chunk masks of the scale image: one word per 32 x 32 chunk, (h/32) rows of (w/32).
inline size_t cmask_words(int w, int h) { return (size_t)((w + 31) / 32) * (size_t)((h + 31) / 32); }
// Per chunk: the mask word and 32 unit masks (one byte per scale: bit u set
// where columns 4u .. 4u + 3 of the chunk hold a pixel of the scale).
inline size_t cmask_bytes(int w, int h) { return align_up(36 * cmask_words(w, h), 256); }
#ifdef __CUDACC__
// The unit masks of an image's chunks (after its mask words, counted on w).
__device__ __forceinline__ uint8_t *chunk_units(const ImgDesc &d)
{
    return (uint8_t *)(d.cmask + (size_t)((d.w + 31) / 32) * ((d.h + 31) / 32));
}
#endif

// Stage launchers over a batch (fd4_scale.cu, fd4_fed.cu); nonzero on a CUDA error.
int launch_select_batch(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                        cudaStream_t st);
int launch_tensor_batch(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                        cudaStream_t st);
// nfield = N at each pixel's selected scale, one strip-walking launch per scale (fd4_tensor.cu).
int launch_tensor_strips(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                         cudaStream_t st);
// Crease segments of one image (fd4_creases.cu); d_ws holds the d / nu field.
int launch_creases(const float *d_u, int w, int h, int pitch, float sigma, int mode, float *d_segs, int *d_keys,
                   int max_segs, int *d_count, void *d_ws, cudaStream_t st);
// IFOD tensor (1, 0, g, g) of every image of a batch from u (fd4_tensor.cu).
int launch_ifod_tensor(const HostBatch &B, float sigma, const fd4_params &p, cudaStream_t st);
// Scale-image post-processing of every image of a batch from idx, vmax and u
// (fd4_postproc.cu): nfield, idx2 and idx are written.
int launch_postprocess_batch(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                             cudaStream_t st);
// Selection planes of every scale and each image's max S^2, one strip-walking
// launch per scale (fd4_tensor.cu); B.max_s2 must be cleared first.
int launch_select_strips(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                         cudaStream_t st);
// Schedule of the FED kernels (no effect on the result beyond FP32 rounding):
// explicit steps per launch (1: k_fed_step; 2, 4: the TMA quad kernel under the
// natural boundary; 3 and the periodic boundary: k_fed_fused<S>), and for the
// TMA kernel its region height (64 or 32 rows of 64 columns) and the row
// quads each thread owns (1 or 2).
struct FedSched {
    int steps, rows, quads;
};
constexpr FedSched kDefaultSched = {2, 64, 2};
FedSched resolve_sched(const fd4_params &p);  // zero fields of p take the default
// n FED steps on every image.  end_parity == nullptr: the result ends in
// ImgDesc::u (copied back from the FED plane after an odd number of launches);
// otherwise nothing is copied and *end_parity = 1 where it ends in ImgDesc::tmp.
int launch_fed_batch(const HostBatch &B, const double *h_tau, int n, int boundary, const FedSched &sch,
                     cudaStream_t st, int *end_parity = nullptr);
// Copies every image's FED plane (ImgDesc::tmp) into ImgDesc::u.
int launch_copy_back_batch(const HostBatch &B, cudaStream_t st);
int launch_select_tiles(const ImgDesc &d, const int *list, const int *count, const float *h_sigmas, int n_sigma,
                        const fd4_params &p, cudaStream_t st);
// Sets the shared-memory attributes of every kernel (call before stream capture).
int prepare_scale_kernels();
int prepare_tensor_kernels();
int prepare_fed_kernels();
int launch_copy_in_batch(const HostBatch &B, cudaStream_t st);
int launch_put_descs(const ImgDesc *h_descs, int n, ImgDesc *d_table, cudaStream_t st);
// TMA staging of the FED kernel (fd4_fed_tma.cu): bytes of one image's maps, the
// writer of a batch's map table (each descriptor's maps field points into it),
// one launch of k <= S steps (region height and quads per thread from sch),
// and the kernels' shared-memory attributes.
size_t tma_maps_bytes();
int launch_put_maps(const ImgDesc *h_descs, int n, void *d_table, cudaStream_t st);
template <int S>
int launch_fed_tma(const HostBatch &B, const double *tau, int k, int parity, const FedSched &sch, cudaStream_t st);
int prepare_tma_kernels();

// Single-image launchers used by the per-image entry points.
int launch_select(const float *d_img, int w, int h, int pitch, const float *h_sigmas,
                  int n_sigma, const fd4_params &p, uint8_t *d_idx, float *d_vmax,
                  char *ws, cudaStream_t st);
int launch_tensor(const float *d_u, int w, int h, int pitch, const uint8_t *d_idx,
                  const float *h_sigmas, int n_sigma, const fd4_params &p, float *d_tensor,
                  char *ws, cudaStream_t st);
int launch_fed_cycle(float *d_u, int w, int h, int pitch, const float *d_tensor,
                     const double *h_tau, int n, int boundary, const FedSched &sch, char *ws, cudaStream_t st);

}  // namespace fd4
