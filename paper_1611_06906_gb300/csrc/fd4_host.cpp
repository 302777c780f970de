// Host side of the fd4 C ABI: parameter defaults, FED step table, Gaussian
// taps, argument validation, workspace layout and the entry points, which
// validate and then enqueue the device kernels (fd4_scale.cu, fd4_fed.cu).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

#include "fd4_internal.h"

using namespace fd4;

extern "C" void fd4_default_params(fd4_params *p)
{
    if (!p) return;
    p->lambda = 0.005f;   // Sec. 4.1 and 4.3
    p->rho = 0.5f;        // Sec. 3.1
    p->beta = 0.5f;       // Sec. 3.3
    p->c = 0.0f;          // auto: half the maximum of S (Sec. 3.3)
    p->gamma = 1.0f;      // sigma^2 normalisation (Sec. 3.3)
    p->tau_max = 0.05f;   // Sec. 3.5
    p->mode = FD4_BOTH;   // "enhancing both ridges and valleys" (Sec. 3.2)
    p->boundary = FD4_BC_NATURAL;
    p->kappa = 0;
    p->grad_norm_squared = 0;
    p->reselect_each_cycle = 0;
    p->postprocess_scales = 0;
    p->theta = 0.2f;
    p->model = FD4_MODEL_MAFOD;
    p->ifod_sigma = 1.0f;
    p->fed_steps_per_launch = 0;
    p->fed_tile_rows = 0;
    p->fed_quads_per_thread = 0;
}

extern "C" const char *fd4_strerror(int s)
{
    switch (s) {
    case FD4_OK: return "ok";
    case FD4_ERR_BAD_ARG: return "bad argument";
    case FD4_ERR_UNSTABLE_TAU: return "FED step sizes exceed the stability limit";
    case FD4_ERR_TOO_MANY_SIGMAS: return "too many scales";
    case FD4_ERR_PITCH: return "row pitch must be >= width and a multiple of 4";
    case FD4_ERR_WS_TOO_SMALL: return "workspace too small";
    case FD4_ERR_TIMEOUT: return "device-side wait timed out";
    case FD4_ERR_CUDA: return "CUDA runtime error";
    case FD4_ERR_ALIGN: return "device pointer not 16-byte aligned";
    case FD4_ERR_SIGMA_RANGE: return "scales must be increasing and in (0, 12]";
    case FD4_ERR_NOT_IMPLEMENTED: return "not implemented";
    default: return "unknown status";
    }
}

extern "C" int fd4_version(void) { return 100; }

// ---------------------------------------------------------------------------
// FED step table (Sec. 3.5, Eq. 22-23) and the kappa ordering.

static double growth_bound(const std::vector<double> &tau_nat, int kappa)
{
    // A(kappa) = max_j PRE_j * SUF_j with PRE_j = max_p |prod_{l<j} f_l(p)| and
    // SUF_j = max_q |prod_{l>=j} f_l(q)|, f_l(p) = 1 - tau_{kappa l mod n} p.
    const int n = (int)tau_nat.size();
    const int NP = 4096;
    std::vector<double> pre(n + 1, 0.0), suf(n + 1, 0.0), run(n + 1);
    for (int ip = 0; ip < NP; ++ip) {
        const double p = 34.0 * ip / (NP - 1);
        run[0] = 1.0;
        for (int l = 0; l < n; ++l)
            run[l + 1] = run[l] * (1.0 - tau_nat[(size_t)((long long)kappa * l % n)] * p);
        for (int j = 0; j <= n; ++j)
            pre[j] = std::fmax(pre[j], std::fabs(run[j]));
        double tail = 1.0;
        suf[n] = std::fmax(suf[n], 1.0);
        for (int j = n - 1; j >= 0; --j) {
            tail *= 1.0 - tau_nat[(size_t)((long long)kappa * j % n)] * p;
            suf[j] = std::fmax(suf[j], std::fabs(tail));
        }
    }
    double a = 0.0;
    for (int j = 0; j <= n; ++j)
        a = std::fmax(a, pre[j] * suf[j]);
    return a;
}

static int gcd_int(int a, int b)
{
    while (b != 0) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

extern "C" int fd4_fed_taus(double T, int M, double tau_max, int n_in, int kappa_in,
                            double *tau_out, int tau_cap, int *n_out, int *kappa_out)
{
    if (!tau_out || !n_out || !(T > 0.0) || M <= 0 || !(tau_max > 0.0) || n_in < 0 || kappa_in < 0)
        return FD4_ERR_BAD_ARG;
    if (tau_max > 1.0 / 17.0 + 1e-12)  // Gershgorin bound of Sec. 3.4 at unit spacing
        return FD4_ERR_UNSTABLE_TAU;
    int n = n_in;
    if (n == 0) {
        const double v = -0.5 + 0.5 * std::sqrt(1.0 + 12.0 * T / (M * tau_max));
        n = (int)std::ceil(v);
        if (n < 1) n = 1;
    }
    if (n > FD4_MAX_FED_STEPS || n > tau_cap)
        return FD4_ERR_BAD_ARG;
    const double nn = (double)n * (double)n + (double)n;
    if (3.0 * T / (M * nn) > tau_max * (1.0 + 1e-12))
        return FD4_ERR_UNSTABLE_TAU;
    std::vector<double> nat(n);
    for (int i = 0; i < n; ++i) {
        const double c = std::cos(M_PI * (2.0 * i + 1.0) / (4.0 * n + 2.0));
        nat[i] = 3.0 * T / (2.0 * M * nn * c * c);
    }
    int kappa = kappa_in;
    if (kappa == 0) {
        double best = HUGE_VAL;
        kappa = 1;
        const int kmax = n > 1 ? n - 1 : 1;
        for (int k = 1; k <= kmax; ++k) {
            if (n > 1 && gcd_int(k, n) != 1) continue;
            const double a = growth_bound(nat, k);
            if (a < best) {
                best = a;
                kappa = k;
            }
        }
    } else if (n > 1 && gcd_int(kappa % n, n) != 1) {
        return FD4_ERR_BAD_ARG;
    }
    for (int i = 0; i < n; ++i)
        tau_out[i] = nat[(size_t)((long long)kappa * i % n)];
    *n_out = n;
    if (kappa_out) *kappa_out = kappa;
    return FD4_OK;
}

// ---------------------------------------------------------------------------
// Gaussian taps.  Sampled at integer offsets, radius ceil(4 sigma): the
// smoothing kernel sums to one, the first-derivative kernel maps the ramp x to
// 1, the second-derivative kernel has zero sum and maps x^2/2 to 1.

int fd4::gauss_taps(double sigma, GaussTaps *t)
{
    const int r = (int)std::ceil(4.0 * sigma);
    if (!(sigma > 0.0) || r > kMaxRadius) return FD4_ERR_SIGMA_RANGE;
    t->r = r;
    const int n = 2 * r + 1;
    std::vector<double> g(n), d1(n), d2(n);
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    double sg = 0.0;
    for (int i = 0; i < n; ++i) {
        const double x = i - r;
        g[i] = std::exp(-x * x * inv2s2);
        sg += g[i];
    }
    double m2 = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double x = i - r;
        g[i] /= sg;
        d1[i] = x * g[i];                          // proportional to -G'(-x)
        m2 += x * d1[i];
        d2[i] = (x * x - sigma * sigma) * g[i];    // proportional to G''(x)
        s2 += d2[i];
    }
    double q = 0.0;
    for (int i = 0; i < n; ++i) {
        const double x = i - r;
        d1[i] /= m2;
        d2[i] -= s2 * g[i];
        q += 0.5 * x * x * d2[i];
    }
    for (int i = 0; i < n; ++i) {
        t->w0[i] = (float)g[i];
        t->w1[i] = (float)d1[i];
        t->w2[i] = (float)(d2[i] / q);
    }
    return FD4_OK;
}

int fd4::rho_taps(double rho, RhoTaps *t)
{
    const int r = (int)std::ceil(4.0 * rho);
    if (!(rho > 0.0) || r > kMaxRhoRadius) return FD4_ERR_BAD_ARG;
    t->r = r;
    std::vector<double> g(2 * r + 1);
    double s = 0.0;
    for (int i = 0; i <= 2 * r; ++i) {
        const double x = i - r;
        g[i] = std::exp(-x * x / (2.0 * rho * rho));
        s += g[i];
    }
    for (int i = 0; i <= 2 * r; ++i)
        t->w0[i] = (float)(g[i] / s);
    return FD4_OK;
}

// ---------------------------------------------------------------------------
// Validation and workspace layout.

int fd4::check_image(const void *d, int w, int h, int pitch)
{
    if (!d || w < 3 || h < 3) return FD4_ERR_BAD_ARG;
    if (pitch < w || (pitch & 3) != 0) return FD4_ERR_PITCH;
    if (((uintptr_t)d & 15u) != 0) return FD4_ERR_ALIGN;
    if ((double)h * (double)pitch * 16.0 > 9.0e18) return FD4_ERR_BAD_ARG;
    return FD4_OK;
}

int fd4::check_sigmas(const float *s, int n)
{
    if (!s || n <= 0) return FD4_ERR_BAD_ARG;
    if (n > FD4_MAX_SIGMAS) return FD4_ERR_TOO_MANY_SIGMAS;
    for (int i = 0; i < n; ++i) {
        if (!(s[i] > 0.0f) || !(s[i] <= FD4_MAX_SIGMA)) return FD4_ERR_SIGMA_RANGE;
        if (i > 0 && !(s[i] > s[i - 1])) return FD4_ERR_SIGMA_RANGE;
    }
    return FD4_OK;
}

void fd4::resolve_params(const fd4_params *in, fd4_params *out)
{
    if (in) *out = *in;
    else fd4_default_params(out);
}

static int check_params(const fd4_params &p)
{
    if (!(p.lambda > 0.0f) || !(p.rho > 0.0f) || !(p.beta > 0.0f) || !(p.gamma >= 0.0f))
        return FD4_ERR_BAD_ARG;
    if ((int)std::ceil(4.0 * p.rho) > kMaxRhoRadius) return FD4_ERR_BAD_ARG;
    if (p.mode < FD4_RIDGE || p.mode > FD4_BOTH) return FD4_ERR_BAD_ARG;
    if (p.boundary != FD4_BC_NATURAL && p.boundary != FD4_BC_PERIODIC) return FD4_ERR_BAD_ARG;
    if (!(p.c >= 0.0f) && !(p.c < 0.0f)) return FD4_ERR_BAD_ARG;  // NaN
    if (p.reselect_each_cycle != 0 && p.reselect_each_cycle != 1) return FD4_ERR_BAD_ARG;
    if (p.postprocess_scales != 0 && p.postprocess_scales != 1) return FD4_ERR_BAD_ARG;
    if (!(p.theta >= 0.0f && p.theta <= 1.0f)) return FD4_ERR_BAD_ARG;
    if (p.model != FD4_MODEL_MAFOD && p.model != FD4_MODEL_IFOD) return FD4_ERR_BAD_ARG;
    if (!(p.ifod_sigma > 0.0f && p.ifod_sigma <= FD4_MAX_SIGMA)) return FD4_ERR_BAD_ARG;
    return FD4_OK;
}

size_t fd4::plane_bytes(int h, int pitch, size_t elem)
{
    return align_up((size_t)h * (size_t)pitch * elem, 256);
}

size_t fd4::ws_select_bytes(int h, int pitch, int n_sigma)
{
    return kHeaderBytes + 2 * (size_t)n_sigma * plane_bytes(h, pitch, 4);
}

// tensor build: header | N field | chunk masks of the scale image
size_t fd4::ws_tensor_bytes(int h, int pitch) { return kHeaderBytes + plane_bytes(h, pitch, 16) + cmask_bytes(pitch, h); }

size_t fd4::ws_fed_bytes(int h, int pitch) { return kHeaderBytes + plane_bytes(h, pitch, 4); }

// filter: sigma* (u8) | tensor field (float4) | chunk masks | stage workspace shared by the stages
size_t fd4::ws_filter_bytes(int h, int pitch, int n_sigma)
{
    size_t stage = ws_select_bytes(h, pitch, n_sigma);
    if (ws_tensor_bytes(h, pitch) > stage) stage = ws_tensor_bytes(h, pitch);
    if (ws_fed_bytes(h, pitch) > stage) stage = ws_fed_bytes(h, pitch);
    return plane_bytes(h, pitch, 1) + plane_bytes(h, pitch, 16) + cmask_bytes(pitch, h) + stage;
}

extern "C" size_t fd4_workspace_bytes(int op, int w, int h, int n_sigma)
{
    if (w < 1 || h < 1 || n_sigma < 0) return 0;
    const int pitch = (int)align_up((size_t)w, 4);
    switch (op) {
    case FD4_OP_SELECT_SCALES: return ws_select_bytes(h, pitch, n_sigma);
    case FD4_OP_BUILD_TENSOR: return ws_tensor_bytes(h, pitch);
    case FD4_OP_FED_CYCLE: return ws_fed_bytes(h, pitch);
    case FD4_OP_FILTER: return ws_filter_bytes(h, pitch, n_sigma);
    case FD4_OP_POSTPROCESS: return plane_bytes(h, pitch, 16) + plane_bytes(h, pitch, 1);
    case FD4_OP_CREASES: return plane_bytes(h, pitch, 8);
    default: return 0;
    }
}

static int ws_ok(const void *ws, size_t have, size_t need)
{
    if (!ws) return FD4_ERR_BAD_ARG;
    if (((uintptr_t)ws & 255u) != 0) return FD4_ERR_ALIGN;
    return have >= need ? FD4_OK : FD4_ERR_WS_TOO_SMALL;
}

static int cuda_status(int e) { return e == 0 ? FD4_OK : FD4_ERR_CUDA; }

// ---------------------------------------------------------------------------
// Entry points.

extern "C" int fd4_select_scales(const float *d_img, int w, int h, int pitch, const float *h_sigmas,
                                 int n_sigma, const fd4_params *params, uint8_t *d_sigma_idx,
                                 float *d_vmax, void *d_ws, size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    fd4_params p;
    resolve_params(params, &p);
    if ((rc = check_image(d_img, w, h, pitch)) != FD4_OK) return rc;
    if ((rc = check_sigmas(h_sigmas, n_sigma)) != FD4_OK) return rc;
    if ((rc = check_params(p)) != FD4_OK) return rc;
    if (!d_sigma_idx) return FD4_ERR_BAD_ARG;
    if (d_vmax && ((uintptr_t)d_vmax & 15u)) return FD4_ERR_ALIGN;
    if ((rc = ws_ok(d_ws, ws_bytes, ws_select_bytes(h, pitch, n_sigma))) != FD4_OK) return rc;
    return cuda_status(launch_select(d_img, w, h, pitch, h_sigmas, n_sigma, p, d_sigma_idx, d_vmax,
                                     (char *)d_ws, (cudaStream_t)stream));
}

extern "C" int fd4_postprocess_scales(const float *d_u, int w, int h, int pitch, uint8_t *d_sigma_idx,
                                      const float *d_vmax, const float *h_sigmas, int n_sigma,
                                      const fd4_params *params, void *d_ws, size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    fd4_params p;
    resolve_params(params, &p);
    if ((rc = check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if ((rc = check_sigmas(h_sigmas, n_sigma)) != FD4_OK) return rc;
    if ((rc = check_params(p)) != FD4_OK) return rc;
    if (!d_sigma_idx || !d_vmax) return FD4_ERR_BAD_ARG;
    if ((uintptr_t)d_vmax & 3u) return FD4_ERR_ALIGN;
    const size_t p16 = plane_bytes(h, pitch, 16);
    if ((rc = ws_ok(d_ws, ws_bytes, p16 + plane_bytes(h, pitch, 1))) != FD4_OK) return rc;
    // workspace: [N at the selected scales | second index plane]
    ImgDesc d{};
    d.u = const_cast<float *>(d_u);  // read only
    d.idx = d_sigma_idx;
    d.vmax = const_cast<float *>(d_vmax);  // read only
    d.nfield = (float4 *)d_ws;
    d.idx2 = (uint8_t *)d_ws + p16;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    return cuda_status(launch_postprocess_batch(single_batch(d), h_sigmas, n_sigma, p, (cudaStream_t)stream));
}

extern "C" int fd4_extract_creases(const float *d_u, int w, int h, int pitch, float sigma, int mode,
                                   float *d_segs, int *d_keys, int max_segs, int *d_count, void *d_ws,
                                   size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    if ((rc = check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if (!(sigma > 0.0f && sigma <= 4.0f) || mode < FD4_RIDGE || mode > FD4_BOTH) return FD4_ERR_BAD_ARG;
    if (!d_segs || !d_keys || !d_count || max_segs < 0) return FD4_ERR_BAD_ARG;
    if ((uintptr_t)d_segs & 15u) return FD4_ERR_ALIGN;
    if ((rc = ws_ok(d_ws, ws_bytes, plane_bytes(h, pitch, 8))) != FD4_OK) return rc;
    return cuda_status(launch_creases(d_u, w, h, pitch, sigma, mode, d_segs, d_keys, max_segs, d_count, d_ws,
                                      (cudaStream_t)stream));
}

extern "C" int fd4_build_tensor_ifod(const float *d_u, int w, int h, int pitch, const fd4_params *params,
                                     float *d_tensor, fd4_stream_t stream)
{
    int rc;
    fd4_params p;
    resolve_params(params, &p);
    if ((rc = check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if ((rc = check_params(p)) != FD4_OK) return rc;
    if (!d_tensor) return FD4_ERR_BAD_ARG;
    if ((uintptr_t)d_tensor & 15u) return FD4_ERR_ALIGN;
    ImgDesc d{};
    d.u = const_cast<float *>(d_u);  // read only
    d.tensor = (float4 *)d_tensor;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    return cuda_status(launch_ifod_tensor(single_batch(d), p.ifod_sigma, p, (cudaStream_t)stream));
}

extern "C" int fd4_build_tensor(const float *d_u, int w, int h, int pitch, const uint8_t *d_sigma_idx,
                                const float *h_sigmas, int n_sigma, const fd4_params *params,
                                float *d_tensor, void *d_ws, size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    fd4_params p;
    resolve_params(params, &p);
    if ((rc = check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if ((rc = check_sigmas(h_sigmas, n_sigma)) != FD4_OK) return rc;
    if ((rc = check_params(p)) != FD4_OK) return rc;
    if (!d_sigma_idx || !d_tensor) return FD4_ERR_BAD_ARG;
    if ((uintptr_t)d_tensor & 15u) return FD4_ERR_ALIGN;
    if ((rc = ws_ok(d_ws, ws_bytes, ws_tensor_bytes(h, pitch))) != FD4_OK) return rc;
    return cuda_status(launch_tensor(d_u, w, h, pitch, d_sigma_idx, h_sigmas, n_sigma, p, d_tensor,
                                     (char *)d_ws, (cudaStream_t)stream));
}

extern "C" int fd4_fed_cycle(float *d_u, int w, int h, int pitch, const float *d_tensor,
                             const double *h_tau, int n, int boundary, void *d_ws, size_t ws_bytes,
                             fd4_stream_t stream)
{
    int rc;
    if ((rc = check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if (!d_tensor || !h_tau || n < 1 || n > FD4_MAX_FED_STEPS) return FD4_ERR_BAD_ARG;
    if ((uintptr_t)d_tensor & 15u) return FD4_ERR_ALIGN;
    if (boundary != FD4_BC_NATURAL && boundary != FD4_BC_PERIODIC) return FD4_ERR_BAD_ARG;
    for (int i = 0; i < n; ++i)
        if (!(h_tau[i] > 0.0) || !(h_tau[i] < 1e6)) return FD4_ERR_BAD_ARG;
    if ((rc = ws_ok(d_ws, ws_bytes, ws_fed_bytes(h, pitch))) != FD4_OK) return rc;
    return cuda_status(launch_fed_cycle(d_u, w, h, pitch, d_tensor, h_tau, n, boundary, kDefaultSched,
                                        (char *)d_ws, (cudaStream_t)stream));
}

static int check_sched(int steps, int rows, int quads)
{
    if (steps < 0 || steps > 4) return FD4_ERR_BAD_ARG;
    if (rows != 0 && rows != 32 && rows != 64) return FD4_ERR_BAD_ARG;
    if (quads < 0 || quads > 2) return FD4_ERR_BAD_ARG;
    return FD4_OK;
}

extern "C" int fd4_fed_cycle_sched(float *d_u, int w, int h, int pitch, const float *d_tensor,
                                   const double *h_tau, int n, int boundary, int steps_per_launch, int tile_rows,
                                   int quads_per_thread, void *d_ws, size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    if ((rc = check_sched(steps_per_launch, tile_rows, quads_per_thread)) != FD4_OK) return rc;
    if ((rc = check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if (!d_tensor || !h_tau || n < 1 || n > FD4_MAX_FED_STEPS) return FD4_ERR_BAD_ARG;
    if ((uintptr_t)d_tensor & 15u) return FD4_ERR_ALIGN;
    if (boundary != FD4_BC_NATURAL && boundary != FD4_BC_PERIODIC) return FD4_ERR_BAD_ARG;
    for (int i = 0; i < n; ++i)
        if (!(h_tau[i] > 0.0) || !(h_tau[i] < 1e6)) return FD4_ERR_BAD_ARG;
    if ((rc = ws_ok(d_ws, ws_bytes, ws_fed_bytes(h, pitch))) != FD4_OK) return rc;
    fd4_params p;
    fd4_default_params(&p);
    p.fed_steps_per_launch = steps_per_launch;
    p.fed_tile_rows = tile_rows;
    p.fed_quads_per_thread = quads_per_thread;
    return cuda_status(launch_fed_cycle(d_u, w, h, pitch, d_tensor, h_tau, n, boundary, resolve_sched(p),
                                        (char *)d_ws, (cudaStream_t)stream));
}

// The filter schedule on a batch: selection (unless given), input copy, then M
// cycles of tensor build and FED cycle.  Everything is enqueued on `st`.
// The tensor field of one cycle: MAFOD's at the selected scales, or IFOD's.
static int launch_cycle_tensor(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                               cudaStream_t st)
{
    if (p.model == FD4_MODEL_IFOD) return launch_ifod_tensor(B, p.ifod_sigma, p, st);
    return launch_tensor_batch(B, h_sigmas, n_sigma, p, st);
}

// The batch as the selection sees it when it re-selects on the current image:
// every descriptor's input is the image being filtered (u).  Single images
// carry the descriptor inline; batches have a second device table for it.
static HostBatch current_view(const HostBatch &B)
{
    HostBatch V = B;
    if (B.I.table) V.I.table = B.table_u;
    else V.I.one.in = V.I.one.u;
    return V;
}

static int enqueue_filter(const HostBatch &B, const float *h_sigmas, int n_sigma, const fd4_params &p,
                          const double *tau, int n, int M, int sigma_given, cudaStream_t st,
                          int stages = FD4_STAGES_ALL)
{
    const FedSched sch = resolve_sched(p);
    const bool mafod = p.model == FD4_MODEL_MAFOD;  // IFOD selects no scales
    if (mafod && (stages & FD4_STAGE_SELECT) && !sigma_given && launch_select_batch(B, h_sigmas, n_sigma, p, st))
        return FD4_ERR_CUDA;
    if ((stages & FD4_STAGE_COPY) && launch_copy_in_batch(B, st)) return FD4_ERR_CUDA;
    // the post-processing reads u (the strips' N at the selected scales), so the
    // first one follows the copy of the input into u; a schedule without that
    // copy (a stage-split graph) selects without post-processing
    const bool post = mafod && p.postprocess_scales && !sigma_given && (stages & FD4_STAGE_SELECT) &&
                      (stages & FD4_STAGE_COPY);
    if (post && launch_postprocess_batch(B, h_sigmas, n_sigma, p, st)) return FD4_ERR_CUDA;
    const bool reselect = mafod && p.reselect_each_cycle && !sigma_given && (stages & FD4_STAGE_SELECT);
    // A FED cycle of an odd number of launches ends in the FED plane.  Where
    // the batch has the table with u and that plane exchanged, the next cycle
    // runs on it (its tensor build reads the plane, its FED steps end in u), and
    // the result is copied back at most once, after the last cycle.  Without
    // re-selection the scale image, and with it the chunk masks, stay those of
    // the first cycle.
    const bool alternate = B.table_sw != nullptr && !reselect;
    int view = 0;  // 1: the current image lies in the FED plane
    for (int k = 0; k < M; ++k) {
        if (k > 0 && reselect && launch_select_batch(current_view(B), h_sigmas, n_sigma, p, st))
            return FD4_ERR_CUDA;
        if (k > 0 && reselect && post && launch_postprocess_batch(B, h_sigmas, n_sigma, p, st))
            return FD4_ERR_CUDA;
        HostBatch V = B;
        if (view) V.I.table = B.table_sw;
        V.cmask_fresh = k > 0 && !reselect;
        if ((stages & FD4_STAGE_TENSOR) && launch_cycle_tensor(V, h_sigmas, n_sigma, p, st)) return FD4_ERR_CUDA;
        int end = 0;
        if ((stages & FD4_STAGE_FED) && launch_fed_batch(V, tau, n, p.boundary, sch, st, alternate ? &end : nullptr))
            return FD4_ERR_CUDA;
        view ^= end;
    }
    if (view && launch_copy_back_batch(B, st)) return FD4_ERR_CUDA;
    return FD4_OK;
}

// Whether the filter's FED schedule runs the TMA kernel (2 or 4 steps per
// launch under the natural boundary): its tensor builds then write the FED
// coefficient planes that kernel reads instead of the float4 tensor field.
static bool fed_reads_coef(const fd4_params &p)
{
    const FedSched s = resolve_sched(p);
    return (s.steps == 2 || s.steps == 4) && p.boundary == FD4_BC_NATURAL;
}

static int check_steps(const fd4_params &p)
{
    return check_sched(p.fed_steps_per_launch, p.fed_tile_rows, p.fed_quads_per_thread);
}

extern "C" int fd4_filter(const float *d_in, float *d_out, int w, int h, int pitch,
                          const float *h_sigmas, int n_sigma, const fd4_params *params, double T,
                          int M, int n_in, uint8_t *d_sigma_idx, int sigma_given, void *d_ws,
                          size_t ws_bytes, fd4_stream_t stream)
{
    int rc;
    fd4_params p;
    resolve_params(params, &p);
    if ((rc = check_image(d_in, w, h, pitch)) != FD4_OK) return rc;
    if ((rc = check_image(d_out, w, h, pitch)) != FD4_OK) return rc;
    if ((rc = check_sigmas(h_sigmas, n_sigma)) != FD4_OK) return rc;
    if ((rc = check_params(p)) != FD4_OK) return rc;
    if ((rc = check_steps(p)) != FD4_OK) return rc;
    if (sigma_given && !d_sigma_idx) return FD4_ERR_BAD_ARG;
    if ((rc = ws_ok(d_ws, ws_bytes, ws_filter_bytes(h, pitch, n_sigma))) != FD4_OK) return rc;
    std::vector<double> tau(FD4_MAX_FED_STEPS);
    int n = 0;
    if ((rc = fd4_fed_taus(T, M, p.tau_max, n_in, p.kappa, tau.data(), FD4_MAX_FED_STEPS, &n, nullptr)) != FD4_OK)
        return rc;

    // [sigma* plane | tensor plane | stage workspace = header + scratch]; the
    // stages run in order on one stream, so they share the scratch.
    char *ws = (char *)d_ws;
    uint32_t *cmask = (uint32_t *)(ws + plane_bytes(h, pitch, 1) + plane_bytes(h, pitch, 16));
    char *sws = (char *)cmask + cmask_bytes(pitch, h);
    char *scratch = sws + kHeaderBytes;
    const size_t pb = plane_bytes(h, pitch, 4);
    ImgDesc d{};
    d.in = d_in;
    d.u = d_out;
    d.tmp = (float *)scratch;
    d.vp = (float *)scratch;
    d.s2 = (float *)(scratch + (size_t)n_sigma * pb);
    d.nfield = (float4 *)scratch;
    d.tensor = (float4 *)(ws + plane_bytes(h, pitch, 1));
    d.idx = d_sigma_idx ? d_sigma_idx : (uint8_t *)ws;
    // post-processing: V_max (4 B per pixel) and the second index plane (1 B)
    // packed into the tensor plane (16 B per pixel), which no stage uses
    // between a selection and the cycle's tensor build
    d.vmax = (p.model == FD4_MODEL_MAFOD && p.postprocess_scales && !sigma_given) ? (float *)d.tensor : nullptr;
    d.idx2 = (uint8_t *)d.tensor + 4 * (size_t)h * pitch;
    d.max_s2 = &((WsHeader *)sws)->max_s2;
    d.cmask = cmask;
    d.plane = pb / 4;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    HostBatch B = single_batch(d);
    B.fed_soa = fed_reads_coef(p);
    return enqueue_filter(B, h_sigmas, n_sigma, p, tau.data(), n, M, sigma_given, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Batches.  Workspace: [descriptor table | the table with in = u | the table
// with u and the FED plane exchanged | max S^2 words | TMA maps | the exchanged
// table's maps | per image: sigma* plane, tensor plane (float4 tensor field or
// FED coefficient planes), chunk masks, scratch (selection planes / N field
// and FED plane)].

// Scratch of one image: the selection planes (vp, s2) over the whole of it; the
// N field at its start and the FED plane right after the N field, so that the
// current image may lie in the FED plane while a tensor build writes N.
static size_t scratch_bytes(int h, int pitch, int n_sigma)
{
    size_t sc = 2 * (size_t)n_sigma * plane_bytes(h, pitch, 4);
    const size_t nt = plane_bytes(h, pitch, 16) + plane_bytes(h, pitch, 4);
    if (nt > sc) sc = nt;
    return sc;
}

// split (0 < split < n): images [split, n) form a second group whose tile
// numbering restarts at 0 and which B1 describes (B covers [0, split)).
static size_t batch_layout(const fd4_image *imgs, int n, int n_sigma, std::vector<ImgDesc> *descs, char *ws,
                           HostBatch *B, int split = 0, HostBatch *B1 = nullptr, bool post = false)
{
    size_t off = align_up(sizeof(ImgDesc) * (size_t)n, 256);
    const size_t tu_off = off;  // the same descriptors with in = u (re-selection)
    off += align_up(sizeof(ImgDesc) * (size_t)n, 256);
    const size_t tsw_off = off;  // the descriptors with u and tmp exchanged (odd cycles)
    off += align_up(sizeof(ImgDesc) * (size_t)n, 256);
    const size_t ms_off = off;
    off += align_up(sizeof(unsigned) * (size_t)n, 256);
    const size_t maps_off = off;  // TMA tensor maps of the FED kernel, one set per image
    off += align_up(tma_maps_bytes() * (size_t)n, 256);
    // then the same maps with u and tmp exchanged (the exchanged table's)
    off += align_up(tma_maps_bytes() * (size_t)n, 256);
    int t0[kShapes] = {};
    if (descs) descs->resize(n);
    int t_split[kShapes] = {};
    for (int i = 0; i < n; ++i) {
        if (i == split && split > 0)
            for (int s = 0; s < kShapes; ++s) {
                t_split[s] = t0[s];
                t0[s] = 0;
            }
        const fd4_image &im = imgs[i];
        const size_t pb = plane_bytes(im.h, im.pitch, 4);
        const size_t o_idx = off, o_ten = o_idx + plane_bytes(im.h, im.pitch, 1);
        const size_t o_cm = o_ten + plane_bytes(im.h, im.pitch, 16);
        const size_t o_sc = o_cm + cmask_bytes(im.pitch, im.h);
        off = o_sc + scratch_bytes(im.h, im.pitch, n_sigma);
        if (!descs) continue;
        ImgDesc &d = (*descs)[i];
        d = ImgDesc{};
        d.in = im.d_in;
        d.u = im.d_out;
        d.tmp = (float *)(ws + o_sc + plane_bytes(im.h, im.pitch, 16));
        d.vp = (float *)(ws + o_sc);
        d.s2 = (float *)(ws + o_sc + (size_t)n_sigma * pb);
        d.nfield = (float4 *)(ws + o_sc);
        d.tensor = (float4 *)(ws + o_ten);
        d.idx = im.d_sigma_idx ? im.d_sigma_idx : (uint8_t *)(ws + o_idx);
        // post-processing: V_max (4 B per pixel) and the second index plane (1 B)
        // packed into the tensor plane (16 B per pixel)
        d.vmax = post ? (float *)(ws + o_ten) : nullptr;
        d.idx2 = (uint8_t *)(ws + o_ten) + 4 * (size_t)im.h * im.pitch;
        d.max_s2 = (unsigned *)(ws + ms_off) + i;
        d.cmask = (uint32_t *)(ws + o_cm);
        d.maps = ws + maps_off + tma_maps_bytes() * (size_t)i;
        d.plane = pb / 4;
        d.w = im.w;
        d.h = im.h;
        d.pitch = im.pitch;
        for (int s = 0; s < kShapes; ++s) {
            d.t0[s] = t0[s];
            t0[s] += tiles_of(im.w, im.h, s);
        }
    }
    const bool two = split > 0 && split < n;
    if (B) {
        B->I.table = (const ImgDesc *)ws;
        B->I.n = two ? split : n;
        B->I.tiles = 0;
        B->I.one = ImgDesc{};
        B->I.list = nullptr;
        B->I.count = nullptr;
        for (int s = 0; s < kShapes; ++s) B->tiles[s] = two ? t_split[s] : t0[s];
        B->max_s2 = (unsigned *)(ws + ms_off);
        B->n_max_s2 = two ? split : n;
        B->table_u = (const ImgDesc *)(ws + tu_off);
        B->table_sw = (const ImgDesc *)(ws + tsw_off);
        B->has_cmask = true;
        B->cmask_fresh = false;
        B->fed_soa = false;
    }
    if (B1 && two) {
        *B1 = *B;
        B1->I.table = (const ImgDesc *)ws + split;
        B1->I.n = n - split;
        for (int s = 0; s < kShapes; ++s) B1->tiles[s] = t0[s];
        B1->max_s2 = (unsigned *)(ws + ms_off) + split;
        B1->n_max_s2 = n - split;
        B1->table_u = (const ImgDesc *)(ws + tu_off) + split;
        B1->table_sw = (const ImgDesc *)(ws + tsw_off) + split;
    }
    return off;
}

// Split point that balances the pixel counts of the two groups.
static int balanced_split(const fd4_image *imgs, int n)
{
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += (double)imgs[i].w * imgs[i].h;
    double acc = 0.0;
    int best = 1;
    double err = 1e300;
    for (int k = 1; k < n; ++k) {
        acc += (double)imgs[k - 1].w * imgs[k - 1].h;
        const double e = fabs(2.0 * acc - tot);
        if (e < err) {
            err = e;
            best = k;
        }
    }
    return best;
}

extern "C" size_t fd4_batch_workspace_bytes(const fd4_image *h_imgs, int n_images, int n_sigma)
{
    if (!h_imgs || n_images < 1 || n_images > FD4_MAX_BATCH || n_sigma < 0) return 0;
    for (int i = 0; i < n_images; ++i)
        if (h_imgs[i].w < 1 || h_imgs[i].h < 1 || h_imgs[i].pitch < h_imgs[i].w) return 0;
    return batch_layout(h_imgs, n_images, n_sigma, nullptr, nullptr, nullptr);
}

// Validates a batch call and computes its step sizes.
static int batch_prepare(const fd4_image *imgs, int n_images, const float *h_sigmas, int n_sigma,
                         const fd4_params &p, double T, int M, int n_in, int sigma_given, const void *d_ws,
                         size_t ws_bytes, std::vector<double> &tau, int &n)
{
    int rc;
    if (!imgs || n_images < 1 || n_images > FD4_MAX_BATCH) return FD4_ERR_BAD_ARG;
    for (int i = 0; i < n_images; ++i) {
        const fd4_image &im = imgs[i];
        if ((rc = check_image(im.d_in, im.w, im.h, im.pitch)) != FD4_OK) return rc;
        if ((rc = check_image(im.d_out, im.w, im.h, im.pitch)) != FD4_OK) return rc;
        if (sigma_given && !im.d_sigma_idx) return FD4_ERR_BAD_ARG;
    }
    if ((rc = check_sigmas(h_sigmas, n_sigma)) != FD4_OK) return rc;
    if ((rc = check_params(p)) != FD4_OK) return rc;
    if ((rc = check_steps(p)) != FD4_OK) return rc;
    if ((rc = ws_ok(d_ws, ws_bytes, fd4_batch_workspace_bytes(imgs, n_images, n_sigma))) != FD4_OK) return rc;
    tau.assign(FD4_MAX_FED_STEPS, 0.0);
    return fd4_fed_taus(T, M, p.tau_max, n_in, p.kappa, tau.data(), FD4_MAX_FED_STEPS, &n, nullptr);
}

// The device tables of a batch: the descriptors, the FED kernel's tensor maps
// and, when the filter re-selects on the current image, the descriptors with
// in = u (B.table_u); otherwise the descriptors with u and the FED plane
// exchanged (B.table_sw) with their own maps, which follow the batch's maps.
static int put_tables(const std::vector<ImgDesc> &descs, int n, const HostBatch &B, void *d_ws, bool with_u,
                      bool with_sw, cudaStream_t st)
{
    if (launch_put_descs(descs.data(), n, (ImgDesc *)d_ws, st)) return 1;
    if (n > 0 && launch_put_maps(descs.data(), n, (void *)descs[0].maps, st)) return 1;
    if (with_u) {
        std::vector<ImgDesc> du(descs);
        for (ImgDesc &d : du) d.in = d.u;
        if (launch_put_descs(du.data(), n, (ImgDesc *)B.table_u, st)) return 1;
    } else if (with_sw && n > 0 && B.table_sw) {
        std::vector<ImgDesc> dw(descs);
        char *maps_sw = (char *)descs[0].maps + align_up(tma_maps_bytes() * (size_t)n, 256);
        for (int i = 0; i < n; ++i) {
            std::swap(dw[i].u, dw[i].tmp);
            dw[i].maps = maps_sw + tma_maps_bytes() * (size_t)i;
        }
        if (launch_put_descs(dw.data(), n, (ImgDesc *)B.table_sw, st)) return 1;
        if (launch_put_maps(dw.data(), n, (void *)maps_sw, st)) return 1;
    }
    return 0;
}

// Two image groups on two streams: group 1 starts once group 0's first tensor
// build is done, so from then on one group's FED steps (latency-bound) tend to
// run beside the other group's tensor build (FMA-bound).  Each kernel's
// persistent grid takes half the GPU so that kernels of both streams
// co-reside on every SM.  The per-image arithmetic is unchanged.
static int enqueue_batch_two_streams(const fd4_image *imgs, int n_images, const float *h_sigmas, int n_sigma,
                                     const fd4_params &p, const double *tau, int n, int M, int sigma_given,
                                     void *d_ws, cudaStream_t s0, cudaStream_t s1, cudaEvent_t ev_fork,
                                     cudaEvent_t ev_go, cudaEvent_t ev_join)
{
    std::vector<ImgDesc> descs;
    HostBatch B0, B1;
    const int split = balanced_split(imgs, n_images);
    const bool mafod = p.model == FD4_MODEL_MAFOD;
    const bool sel = mafod && !sigma_given;
    const bool post = sel && p.postprocess_scales;
    batch_layout(imgs, n_images, n_sigma, &descs, (char *)d_ws, &B0, split, &B1, post);
    B0.fed_soa = B1.fed_soa = fed_reads_coef(p);
    const bool reselect = sel && p.reselect_each_cycle;
    if (put_tables(descs, n_images, B0, d_ws, reselect, false, s0)) return FD4_ERR_CUDA;
    const FedSched steps = resolve_sched(p);
    if (cudaEventRecord(ev_fork, s0) != cudaSuccess || cudaStreamWaitEvent(s1, ev_fork, 0) != cudaSuccess)
        return FD4_ERR_CUDA;
    set_grid_divisor(2);
    int rc = FD4_OK;
    // group 0: selection, copy, first tensor build; then group 1 may start
    if ((sel && launch_select_batch(B0, h_sigmas, n_sigma, p, s0)) || launch_copy_in_batch(B0, s0) ||
        (post && launch_postprocess_batch(B0, h_sigmas, n_sigma, p, s0)) ||
        launch_cycle_tensor(B0, h_sigmas, n_sigma, p, s0))
        rc = FD4_ERR_CUDA;
    if (rc == FD4_OK && (cudaEventRecord(ev_go, s0) != cudaSuccess || cudaStreamWaitEvent(s1, ev_go, 0) != cudaSuccess))
        rc = FD4_ERR_CUDA;
    if (rc == FD4_OK && ((sel && launch_select_batch(B1, h_sigmas, n_sigma, p, s1)) ||
                         launch_copy_in_batch(B1, s1) || (post && launch_postprocess_batch(B1, h_sigmas, n_sigma, p, s1))))
        rc = FD4_ERR_CUDA;
    for (int k = 0; k < M && rc == FD4_OK; ++k) {
        if (launch_fed_batch(B0, tau, n, p.boundary, steps, s0)) rc = FD4_ERR_CUDA;
        if (rc == FD4_OK && k + 1 < M && reselect && launch_select_batch(current_view(B0), h_sigmas, n_sigma, p, s0))
            rc = FD4_ERR_CUDA;
        if (rc == FD4_OK && k + 1 < M && reselect && post && launch_postprocess_batch(B0, h_sigmas, n_sigma, p, s0))
            rc = FD4_ERR_CUDA;
        if (rc == FD4_OK && k + 1 < M && launch_cycle_tensor(B0, h_sigmas, n_sigma, p, s0)) rc = FD4_ERR_CUDA;
        if (rc == FD4_OK && k > 0 && reselect && launch_select_batch(current_view(B1), h_sigmas, n_sigma, p, s1))
            rc = FD4_ERR_CUDA;
        if (rc == FD4_OK && k > 0 && reselect && post && launch_postprocess_batch(B1, h_sigmas, n_sigma, p, s1))
            rc = FD4_ERR_CUDA;
        if (rc == FD4_OK && launch_cycle_tensor(B1, h_sigmas, n_sigma, p, s1)) rc = FD4_ERR_CUDA;
        if (rc == FD4_OK && launch_fed_batch(B1, tau, n, p.boundary, steps, s1)) rc = FD4_ERR_CUDA;
    }
    set_grid_divisor(1);
    if (cudaEventRecord(ev_join, s1) != cudaSuccess || cudaStreamWaitEvent(s0, ev_join, 0) != cudaSuccess)
        return FD4_ERR_CUDA;
    return rc;
}

static int enqueue_batch(const fd4_image *imgs, int n_images, const float *h_sigmas, int n_sigma,
                         const fd4_params &p, const double *tau, int n, int M, int sigma_given, void *d_ws,
                         cudaStream_t st, int stages = FD4_STAGES_ALL)
{
    std::vector<ImgDesc> descs;
    HostBatch B;
    const bool sel = p.model == FD4_MODEL_MAFOD && !sigma_given && (stages & FD4_STAGE_SELECT);
    const bool post = sel && p.postprocess_scales && (stages & FD4_STAGE_COPY);
    batch_layout(imgs, n_images, n_sigma, &descs, (char *)d_ws, &B, 0, nullptr, post);
    B.fed_soa = fed_reads_coef(p);
    const bool reselect = sel && p.reselect_each_cycle;
    // the exchanged table serves cycles that end in the FED plane
    const bool with_sw = !reselect && (stages & FD4_STAGE_FED);
    if (!with_sw) B.table_sw = nullptr;
    if (put_tables(descs, n_images, B, d_ws, reselect, with_sw, st)) return FD4_ERR_CUDA;
    return enqueue_filter(B, h_sigmas, n_sigma, p, tau, n, M, sigma_given, st, stages);
}

extern "C" int fd4_filter_batched(const fd4_image *h_imgs, int n_images, const float *h_sigmas, int n_sigma,
                                  const fd4_params *params, double T, int M, int n_in, int sigma_given,
                                  void *d_ws, size_t ws_bytes, fd4_stream_t stream)
{
    fd4_params p;
    resolve_params(params, &p);
    std::vector<double> tau;
    int n = 0;
    int rc = batch_prepare(h_imgs, n_images, h_sigmas, n_sigma, p, T, M, n_in, sigma_given, d_ws, ws_bytes, tau, n);
    if (rc != FD4_OK) return rc;
    return enqueue_batch(h_imgs, n_images, h_sigmas, n_sigma, p, tau.data(), n, M, sigma_given, d_ws,
                         (cudaStream_t)stream);
}

struct fd4_graph_st {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" int fd4_graph_create(const fd4_image *h_imgs, int n_images, const float *h_sigmas, int n_sigma,
                                const fd4_params *params, double T, int M, int n_in, int sigma_given,
                                int stages, void *d_ws, size_t ws_bytes, fd4_graph *out)
{
    if (!out || (stages & FD4_STAGES_ALL) == 0 || (stages & ~(FD4_STAGES_ALL | FD4_GRAPH_TWO_STREAMS)) != 0)
        return FD4_ERR_BAD_ARG;
    *out = nullptr;
    fd4_params p;
    resolve_params(params, &p);
    std::vector<double> tau;
    int n = 0;
    int rc = batch_prepare(h_imgs, n_images, h_sigmas, n_sigma, p, T, M, n_in, sigma_given, d_ws, ws_bytes, tau, n);
    if (rc != FD4_OK) return rc;
    // kernel attributes are set outside the capture
    if (prepare_scale_kernels() || prepare_fed_kernels()) return FD4_ERR_CUDA;
    const bool two = (stages & FD4_GRAPH_TWO_STREAMS) && n_images >= 2;
    stages &= FD4_STAGES_ALL;
    cudaStream_t s, s1 = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FD4_ERR_CUDA;
    if (two) {
        bool ok = cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 3 && ok; ++i) ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            for (int i = 0; i < 3; ++i)
                if (ev[i]) cudaEventDestroy(ev[i]);
            if (s1) cudaStreamDestroy(s1);
            cudaStreamDestroy(s);
            return FD4_ERR_CUDA;
        }
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(s);
        return FD4_ERR_CUDA;
    }
    if (two && stages == FD4_STAGES_ALL)
        rc = enqueue_batch_two_streams(h_imgs, n_images, h_sigmas, n_sigma, p, tau.data(), n, M, sigma_given, d_ws, s,
                                       s1, ev[0], ev[1], ev[2]);
    else
        rc = enqueue_batch(h_imgs, n_images, h_sigmas, n_sigma, p, tau.data(), n, M, sigma_given, d_ws, s, stages);
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (s1) cudaStreamDestroy(s1);
    for (int i = 0; i < 3; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (rc != FD4_OK || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return rc != FD4_OK ? rc : FD4_ERR_CUDA;
    }
    cudaGraphExec_t e = nullptr;
    if (cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return FD4_ERR_CUDA;
    }
    fd4_graph_st *gs = new fd4_graph_st{g, e};
    *out = gs;
    return FD4_OK;
}

extern "C" int fd4_graph_launch(fd4_graph g, fd4_stream_t stream)
{
    if (!g) return FD4_ERR_BAD_ARG;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? FD4_OK : FD4_ERR_CUDA;
}

extern "C" int fd4_graph_kernel_count(fd4_graph g, int *n_kernels)
{
    if (!g || !n_kernels) return FD4_ERR_BAD_ARG;
    size_t n = 0;
    if (cudaGraphGetNodes(g->graph, nullptr, &n) != cudaSuccess) return FD4_ERR_CUDA;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g->graph, nodes.data(), &n) != cudaSuccess) return FD4_ERR_CUDA;
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) return FD4_ERR_CUDA;
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *n_kernels = k;
    return FD4_OK;
}

extern "C" int fd4_graph_destroy(fd4_graph g)
{
    if (!g) return FD4_ERR_BAD_ARG;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return FD4_OK;
}

extern "C" int fd4_autotune_batched(const fd4_image *h_imgs, int n_images, const float *h_sigmas, int n_sigma,
                                    const fd4_params *params, double T, int M, int n_in, void *d_ws,
                                    size_t ws_bytes, fd4_stream_t stream, fd4_fed_schedule *best,
                                    fd4_fed_schedule *tried)
{
    if (!best) return FD4_ERR_BAD_ARG;
    fd4_params p;
    resolve_params(params, &p);
    std::vector<double> tau;
    int n = 0;
    int rc = batch_prepare(h_imgs, n_images, h_sigmas, n_sigma, p, T, M, n_in, 0, d_ws, ws_bytes, tau, n);
    if (rc != FD4_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<ImgDesc> descs;
    HostBatch B;
    batch_layout(h_imgs, n_images, n_sigma, &descs, (char *)d_ws, &B);
    if (launch_put_descs(descs.data(), n_images, (ImgDesc *)d_ws, st)) return FD4_ERR_CUDA;
    if (n_images > 0 && launch_put_maps(descs.data(), n_images, (void *)descs[0].maps, st)) return FD4_ERR_CUDA;
    B.fed_soa = false;
    if ((p.model == FD4_MODEL_MAFOD && launch_select_batch(B, h_sigmas, n_sigma, p, st)) ||
        launch_copy_in_batch(B, st) || launch_cycle_tensor(B, h_sigmas, n_sigma, p, st))
        return FD4_ERR_CUDA;
    // the candidates: one launch per step, the scalar kernel with 3 steps, and
    // the TMA kernel with 2 or 4 steps on 64- or 32-row regions, 1 or 2 quads
    // per thread (the periodic boundary runs the scalar kernel for 2 and 4)
    const int cand[FD4_AUTOTUNE_CANDIDATES][3] = {{1, 0, 0},  {2, 64, 2}, {2, 64, 1}, {2, 32, 2}, {2, 32, 1},
                                                  {3, 0, 0},  {4, 64, 2}, {4, 64, 1}, {4, 32, 2}, {4, 32, 1}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FD4_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FD4_ERR_CUDA;
    }
    rc = FD4_OK;
    fd4_fed_schedule top{};
    for (int c = 0; c < FD4_AUTOTUNE_CANDIDATES && rc == FD4_OK; ++c) {
        const FedSched sch{cand[c][0], cand[c][1] ? cand[c][1] : kDefaultSched.rows,
                           cand[c][2] ? cand[c][2] : kDefaultSched.quads};
        // the tensor field in the form this candidate reads, as the filter builds it
        fd4_params pc = p;
        pc.fed_steps_per_launch = sch.steps;
        if (fed_reads_coef(pc) != B.fed_soa) {
            B.fed_soa = !B.fed_soa;
            if (launch_cycle_tensor(B, h_sigmas, n_sigma, p, st)) {
                rc = FD4_ERR_CUDA;
                break;
            }
        }
        // one untimed cycle, then the timed one, each without the copy back
        // that the filter's alternating cycles do not make
        int end = 0;
        if (launch_fed_batch(B, tau.data(), n, p.boundary, sch, st, &end) || cudaEventRecord(e0, st) != cudaSuccess ||
            launch_fed_batch(B, tau.data(), n, p.boundary, sch, st, &end) || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) {
            rc = FD4_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const fd4_fed_schedule r{cand[c][0], cand[c][1], cand[c][2], ms};
        if (tried) tried[c] = r;
        if (c == 0 || ms < top.ms) top = r;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == FD4_OK) *best = top;
    return rc;
}
