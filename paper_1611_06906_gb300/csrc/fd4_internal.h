// Internal declarations shared by the fd4 translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fd4.h"

namespace fd4 {

constexpr int kMaxRadius = 64;              // ceil(4 * FD4_MAX_SIGMA)
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

// Launch wrappers (fd4_scale.cu, fd4_fed.cu); they return cudaError_t as int.
int launch_select(const float *d_img, int w, int h, int pitch, const float *h_sigmas,
                  int n_sigma, const fd4_params &p, uint8_t *d_idx, float *d_vmax,
                  char *ws, cudaStream_t st);
int launch_tensor(const float *d_u, int w, int h, int pitch, const uint8_t *d_idx,
                  const float *h_sigmas, int n_sigma, const fd4_params &p, float *d_tensor,
                  char *ws, cudaStream_t st);
int launch_fed_cycle(float *d_u, int w, int h, int pitch, const float *d_tensor,
                     const double *h_tau, int n, int boundary, char *ws, cudaStream_t st);

}  // namespace fd4
