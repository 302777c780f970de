/*
 * FP64 CPU oracle for the MAFOD hot path (multi-scale anisotropic
 * fourth-order diffusion, arXiv:1611.06906).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library: every formula below is
 * written out again from the paper, in double precision, as direct loops.
 *
 * Conventions: images are row-major, index (x, y) = (column, row), pixel
 * value u[y * w + x].  x is the paper's first index i, y its second index j
 * (Sec. 3.4, finite-difference stencils).
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   or_gauss_kernels      pinned: moments, polynomial exactness, continuum limit
 *   or_derivatives        pinned: polynomials, direct 2-D sum, analytic ridge
 *   or_mirror (border)    pinned: scipy.ndimage 'reflect' and numpy
 *                         'symmetric' padding on random images (radius larger
 *                         than the image included), a 4-pixel case by hand
 *   or_select_scales      pinned: width-scale relation, rotation invariance,
 *                         polarity, closed-form eigenvalues
 *   or_build_tensor       pinned: analytic eigen-structure, D:E_k = mu_k E_k,
 *                         ||D|| <= 1, rotation equivariance
 *   or_fed_taus           pinned: sum tau = T/M, n from the paper's own
 *                         parameter sets, cycle polynomial bound
 *   or_apply_P / or_fed_*  pinned: dense P symmetric PSD, P1 = 0, 1'P = 0,
 *                         ||P|| <= 34, periodic biharmonic Fourier multiplier
 *   or_postprocess_*      pinned: hand-built cross-sections along the axes and
 *                         the diagonal (row, column and diagonal means), the
 *                         walk cap, empty mask, isotropic Hessians, a straight
 *                         ridge (one scale per cross-section)
 *   or_crease_field /     pinned: d and nu in closed form on quadratics, the
 *   or_marching_squares   exact zero line of a linear field, both saddle
 *                         resolutions, a straight ridge's centre line, the
 *                         crease-type filter
 *   or_*_ifod             pinned: g = 1 on constants, g in closed form on
 *                         quadratics, g -> 1 as lambda grows (the cycle then
 *                         equals the biharmonic one), mean conservation
 *   or_filter             whole-filter output: parity unpinned beyond the
 *                         invariants above (the paper prints no numeric
 *                         intermediate for it); its cycle schedule (one
 *                         selection, or one per cycle) pinned against the
 *                         composition of the primitives above
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

enum { OR_RIDGE = 0, OR_VALLEY = 1, OR_BOTH = 2 };
enum { OR_NATURAL = 0, OR_PERIODIC = 1 };

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the pixel-row loops from now on (the arithmetic per pixel does
 * not depend on it); used to time the oracle on one core.                   */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gaussian derivative kernels.  The paper regularises with u_sigma = u * G_sigma
 * (Sec. 3.1, Eq. 6, the local normalised Hessian) and takes derivatives of u_sigma;
 * it does not say how the kernel is discretised.  Reading used here: sampled
 * on offsets -r..r with r = ceil(4 sigma); the smoothing kernel sums to 1;
 * the first-derivative kernel is exact on a linear ramp; the second-derivative
 * kernel sums to 0 and is exact on x^2/2.  Weights are correlation weights:
 * out[x] = sum_k w[k] u[x + k].                                               */
int or_gauss_radius(double sigma)
{
    return (int)ceil(4.0 * sigma);
}

void or_gauss_kernels(double sigma, int r, double *w0, double *w1, double *w2)
{
    int n = 2 * r + 1;
    double s2 = sigma * sigma;
    double sum = 0.0;
    for (int k = -r; k <= r; ++k) {
        double g = exp(-(double)(k * k) / (2.0 * s2));
        w0[k + r] = g;
        sum += g;
    }
    for (int i = 0; i < n; ++i)
        w0[i] /= sum;

    /* d/dx G(x) = -x/s2 G(x); as a correlation weight the sign flips, giving
     * k/s2 * G(k).  Normalise so that sum_k w1[k] * k = 1.                    */
    double m2 = 0.0;
    for (int k = -r; k <= r; ++k)
        m2 += (double)k * (double)k / s2 * w0[k + r];
    for (int k = -r; k <= r; ++k)
        w1[k + r] = (double)k / s2 * w0[k + r] / m2;

    /* d2/dx2 G(x) = (x^2/s2^2 - 1/s2) G(x) (even, so no sign flip).           */
    double tot = 0.0;
    for (int k = -r; k <= r; ++k) {
        double v = ((double)(k * k) / (s2 * s2) - 1.0 / s2) * w0[k + r];
        w2[k + r] = v;
        tot += v;
    }
    /* remove the sampled kernel's residual sum along the smoothing kernel    */
    for (int k = -r; k <= r; ++k)
        w2[k + r] -= tot * w0[k + r];
    double q = 0.0;
    for (int k = -r; k <= r; ++k)
        q += 0.5 * (double)(k * k) * w2[k + r];
    for (int k = -r; k <= r; ++k)
        w2[k + r] /= q;
}

/* Half-sample symmetric extension: u[-1-i] = u[i], u[n+i] = u[n-1-i], folded
 * with period 2n so that any offset is defined.  (Boundary handling of the
 * Gaussian convolutions is not stated in the paper; this is our reading.)    */
static int or_mirror(int i, int n)
{
    int p = 2 * n;
    int m = i % p;
    if (m < 0)
        m += p;
    return m < n ? m : p - 1 - m;
}

/* Derivatives of u_sigma = u * G_sigma by separable Gaussian-derivative
 * filtering: a row pass with the smoothing / first / second derivative kernel
 * along x, then a column pass along y.  Any output pointer may be NULL.      */
void or_derivatives(const double *u, int w, int h, double sigma,
                    double *ux, double *uy, double *uxx, double *uxy, double *uyy)
{
    int r = or_gauss_radius(sigma);
    int n = 2 * r + 1;
    double *w0 = malloc(sizeof(double) * n);
    double *w1 = malloc(sizeof(double) * n);
    double *w2 = malloc(sizeof(double) * n);
    or_gauss_kernels(sigma, r, w0, w1, w2);
    size_t np = (size_t)w * h;
    double *r0 = malloc(sizeof(double) * np);
    double *r1 = malloc(sizeof(double) * np);
    double *r2 = malloc(sizeof(double) * np);

#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int k = -r; k <= r; ++k) {
                double v = u[(size_t)y * w + or_mirror(x + k, w)];
                a0 += w0[k + r] * v;
                a1 += w1[k + r] * v;
                a2 += w2[k + r] * v;
            }
            r0[(size_t)y * w + x] = a0;
            r1[(size_t)y * w + x] = a1;
            r2[(size_t)y * w + x] = a2;
        }
    }

#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0, syy = 0.0;
            for (int k = -r; k <= r; ++k) {
                size_t q = (size_t)or_mirror(y + k, h) * w + x;
                sx += w0[k + r] * r1[q];   /* d/dx then smooth in y  */
                sy += w1[k + r] * r0[q];   /* smooth in x then d/dy  */
                sxx += w0[k + r] * r2[q];
                sxy += w1[k + r] * r1[q];
                syy += w2[k + r] * r0[q];
            }
            size_t p = (size_t)y * w + x;
            if (ux) ux[p] = sx;
            if (uy) uy[p] = sy;
            if (uxx) uxx[p] = sxx;
            if (uxy) uxy[p] = sxy;
            if (uyy) uyy[p] = syy;
        }
    }
    free(r0); free(r1); free(r2);
    free(w0); free(w1); free(w2);
}

/* The same derivative by the direct (non-separable) 2-D sum, used only to pin
 * the separable evaluation above.  order_x, order_y in {0,1,2}.              */
void or_derivative_direct(const double *u, int w, int h, double sigma,
                          int order_x, int order_y, double *out)
{
    int r = or_gauss_radius(sigma);
    int n = 2 * r + 1;
    double *wk[3];
    for (int i = 0; i < 3; ++i)
        wk[i] = malloc(sizeof(double) * n);
    or_gauss_kernels(sigma, r, wk[0], wk[1], wk[2]);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double acc = 0.0;
            for (int l = -r; l <= r; ++l)
                for (int k = -r; k <= r; ++k)
                    acc += wk[order_x][k + r] * wk[order_y][l + r] *
                           u[(size_t)or_mirror(y + l, h) * w + or_mirror(x + k, w)];
            out[(size_t)y * w + x] = acc;
        }
    for (int i = 0; i < 3; ++i)
        free(wk[i]);
}

/* ------------------------------------------------------------------------ */
/* Scale selection (Sec. 3.3, Eq. 9 and the text around it).
 * For each sigma: the eigenvalues of sigma^(2 gamma) H(u_sigma), ordered
 * |nu1| <= |nu2| (equal magnitudes: nu2 is the negative one), the structure
 * measure S = sqrt(nu1^2 + nu2^2) and the blob ratio R_B = nu1 / nu2.
 * c = c_in if c_in > 0, else half the maximum of S over all sigma and pixels.
 * V = 0 for the wrong polarity (ridge: nu2 > 0; valley: nu2 < 0; both: never),
 * else exp(-R_B^2 / (2 beta^2)) (1 - exp(-S^2 / (2 c^2))).
 * sigma_idx = argmax over sigma of V, ties to the smaller sigma (the sigmas are
 * given in increasing order).  v_all (nullable) receives V for every sigma as
 * n_sigma planes; v_max (nullable) the maximum.  Returns c.                 */
double or_select_scales(const double *u, int w, int h, const double *sigmas,
                        int n_sigma, int mode, double beta, double c_in,
                        double gamma, uint8_t *sigma_idx, double *v_max,
                        double *v_all)
{
    size_t np = (size_t)w * h;
    double *nu1 = malloc(sizeof(double) * np * n_sigma);
    double *nu2 = malloc(sizeof(double) * np * n_sigma);
    double *a = malloc(sizeof(double) * np);
    double *b = malloc(sizeof(double) * np);
    double *d = malloc(sizeof(double) * np);
    double smax = 0.0;

    for (int s = 0; s < n_sigma; ++s) {
        double sg = sigmas[s];
        double scale = pow(sg, 2.0 * gamma);
        or_derivatives(u, w, h, sg, NULL, NULL, a, b, d);
        for (size_t p = 0; p < np; ++p) {
            double A = scale * a[p], B = scale * b[p], Dd = scale * d[p];
            double m = 0.5 * (A + Dd);
            double rr = hypot(0.5 * (A - Dd), B);
            double lp = m + rr, lm = m - rr;
            double n1, n2;
            if (fabs(lp) > fabs(lm)) { n2 = lp; n1 = lm; }
            else                     { n2 = lm; n1 = lp; }
            nu1[(size_t)s * np + p] = n1;
            nu2[(size_t)s * np + p] = n2;
            double S = sqrt(n1 * n1 + n2 * n2);
            if (S > smax)
                smax = S;
        }
    }

    double c = c_in > 0.0 ? c_in : 0.5 * smax;
    for (size_t p = 0; p < np; ++p) {
        double best = -1.0;
        int arg = 0;
        for (int s = 0; s < n_sigma; ++s) {
            double n1 = nu1[(size_t)s * np + p], n2 = nu2[(size_t)s * np + p];
            double V;
            int wrong = (mode == OR_RIDGE && n2 > 0.0) || (mode == OR_VALLEY && n2 < 0.0);
            if (wrong || c <= 0.0 || n2 == 0.0) {
                V = 0.0;
            } else {
                double RB = n1 / n2;
                double S2 = n1 * n1 + n2 * n2;
                V = exp(-RB * RB / (2.0 * beta * beta)) * (1.0 - exp(-S2 / (2.0 * c * c)));
            }
            if (v_all)
                v_all[(size_t)s * np + p] = V;
            if (V > best) {
                best = V;
                arg = s;
            }
        }
        sigma_idx[p] = (uint8_t)arg;
        if (v_max)
            v_max[p] = best;
    }
    free(nu1); free(nu2); free(a); free(b); free(d);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Scale-image post-processing (Sec. 3.3, the paragraphs after Eq. 9).  Pixels
 * whose vesselness V = max_sigma V_sigma exceeds theta form the vessel mask.
 * For a mask pixel p the vessel cross-section through p is traced along the
 * eigenvector of the Hessian at p's selected scale that belongs to the
 * eigenvalue of largest magnitude (the one the tie rule of or_select_scales
 * calls nu2: on equal magnitudes the negative one), and p takes the scale of
 * the set nearest to the mean scale of the cross-section's pixels.
 * Readings (the paper gives no discretisation): the cross-section is the
 * digital line through p with one pixel per unit step along its major axis
 * (the minor coordinate rounded half up), walked both ways from p while the
 * pixels lie inside the image and the mask, at most cap pixels per side; an
 * isotropic Hessian (equal eigenvalues) gives no direction and p keeps its
 * scale; ties of the nearest scale go to the smaller sigma; all pixels are
 * updated from the scale image as selected, not from updated neighbours; an
 * index outside the scale set (only a caller-given scale image has one) keeps
 * its value and ends a walk like a pixel outside the mask.                   */

/* Unit eigenvector of [a b; b d] for its eigenvalue of largest magnitude
 * (the negative one on a tie); 0 if the eigenvalues are equal.              */
int or_strong_direction(double a, double b, double d, double *ex, double *ey)
{
    double m = 0.5 * (a + d), q = 0.5 * (a - d);
    double r = hypot(q, b);
    if (r == 0.0)
        return 0;
    double vx, vy; /* eigenvector of m + r: a row of [q - r, b; b, -q - r] is orthogonal to it */
    if (q >= 0.0) { vx = q + r; vy = b; }
    else          { vx = b;     vy = r - q; }
    double n = hypot(vx, vy);
    vx /= n;
    vy /= n;
    if (fabs(m + r) > fabs(m - r)) { *ex = vx;  *ey = vy; }
    else                            { *ex = -vy; *ey = vx; }
    return 1;
}

/* The post-processing from given Hessian fields (any positive multiple of the
 * Hessian at each pixel's selected scale gives the same directions).        */
void or_postprocess_core(uint8_t *idx_io, const double *vmax, const double *hxx,
                         const double *hxy, const double *hyy, int w, int h,
                         const double *sigmas, int n_sigma, double theta, int cap)
{
    size_t np = (size_t)w * h;
    uint8_t *out = malloc(np);
    memcpy(out, idx_io, np);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double ex, ey;
            if (idx_io[p] >= n_sigma || !(vmax[p] > theta) ||
                !or_strong_direction(hxx[p], hxy[p], hyy[p], &ex, &ey))
                continue;
            double mx = fmax(fabs(ex), fabs(ey));
            double sx = ex / mx, sy = ey / mx; /* one of them is +-1 */
            double sum = sigmas[idx_io[p]];
            int cnt = 1;
            for (int dir = -1; dir <= 1; dir += 2)
                for (int k = 1; k <= cap; ++k) {
                    int qx = x + (int)floor(dir * k * sx + 0.5);
                    int qy = y + (int)floor(dir * k * sy + 0.5);
                    if (qx < 0 || qy < 0 || qx >= w || qy >= h)
                        break;
                    size_t q = (size_t)qy * w + qx;
                    if (!(vmax[q] > theta) || idx_io[q] >= n_sigma)
                        break;
                    sum += sigmas[idx_io[q]];
                    ++cnt;
                }
            double mean = sum / cnt;
            int arg = 0;
            double best = fabs(sigmas[0] - mean);
            for (int s = 1; s < n_sigma; ++s) {
                double dd = fabs(sigmas[s] - mean);
                if (dd < best) {
                    best = dd;
                    arg = s;
                }
            }
            out[p] = (uint8_t)arg;
        }
    memcpy(idx_io, out, np);
    free(out);
}

/* The post-processing of the scale image selected on u: the Hessian of u_sigma
 * at each pixel's selected scale, the walk capped at the largest kernel radius
 * ceil(4 sigma_max).                                                         */
void or_postprocess_scales(const double *u, int w, int h, uint8_t *idx_io,
                           const double *vmax, const double *sigmas, int n_sigma,
                           double theta)
{
    size_t np = (size_t)w * h;
    double *hxx = calloc(np, sizeof(double));
    double *hxy = calloc(np, sizeof(double));
    double *hyy = calloc(np, sizeof(double));
    double *a = malloc(sizeof(double) * np);
    double *b = malloc(sizeof(double) * np);
    double *d = malloc(sizeof(double) * np);
    for (int s = 0; s < n_sigma; ++s) {
        or_derivatives(u, w, h, sigmas[s], NULL, NULL, a, b, d);
        for (size_t p = 0; p < np; ++p)
            if (idx_io[p] == s) {
                hxx[p] = a[p];
                hxy[p] = b[p];
                hyy[p] = d[p];
            }
    }
    double smax = sigmas[0];
    for (int s = 1; s < n_sigma; ++s)
        if (sigmas[s] > smax)
            smax = sigmas[s];
    or_postprocess_core(idx_io, vmax, hxx, hxy, hyy, w, h, sigmas, n_sigma, theta,
                        or_gauss_radius(smax));
    free(hxx); free(hxy); free(hyy); free(a); free(b); free(d);
}

/* ------------------------------------------------------------------------ */
/* Perona-Malik diffusivity of one eigenvalue with the ridge/valley gating of
 * Sec. 3.2 (Eq. 7 and the paragraph after it).                  */
static double or_mu(double nu, double lambda, int mode)
{
    if (mode == OR_RIDGE && nu >= 0.0)
        return 1.0;
    if (mode == OR_VALLEY && nu <= 0.0)
        return 1.0;
    return 1.0 / (1.0 + nu * nu / (lambda * lambda));
}

/* Fourth-order diffusion tensor field (Sec. 3.1 Eq. 6, Sec. 3.2 Eq. 7-8).
 * N = H(u_sigma*) / sqrt(1 + |grad u_sigma*|), sigma* taken per pixel from
 * sigma_idx (|grad| squared inside the root if grad_sq), N_rho = G_rho * N
 * componentwise, then the eigen-decomposition of N_rho gives e1 (larger
 * eigenvalue nu1) and e2, and mu_i = g(nu_i).  Output per pixel, as four
 * planes: cos(2 theta), sin(2 theta), mu1, mu2 with e1 = (cos theta, sin theta).
 * n_out (nullable) receives N_rho as three planes (xx, xy, yy).             */
void or_build_tensor(const double *u, int w, int h, const uint8_t *sigma_idx,
                     const double *sigmas, int n_sigma, double lambda,
                     double rho, int mode, int grad_sq, double *tensor,
                     double *n_out)
{
    size_t np = (size_t)w * h;
    double *nxx = calloc(np, sizeof(double));
    double *nxy = calloc(np, sizeof(double));
    double *nyy = calloc(np, sizeof(double));
    double *ux = malloc(sizeof(double) * np);
    double *uy = malloc(sizeof(double) * np);
    double *uxx = malloc(sizeof(double) * np);
    double *uxy = malloc(sizeof(double) * np);
    double *uyy = malloc(sizeof(double) * np);

    for (int s = 0; s < n_sigma; ++s) {
        int used = 0;
        for (size_t p = 0; p < np && !used; ++p)
            used = sigma_idx[p] == s;
        if (!used)
            continue;
        or_derivatives(u, w, h, sigmas[s], ux, uy, uxx, uxy, uyy);
        for (size_t p = 0; p < np; ++p) {
            if (sigma_idx[p] != s)
                continue;
            double g2 = ux[p] * ux[p] + uy[p] * uy[p];
            double g = grad_sq ? g2 : sqrt(g2);
            double f = 1.0 / sqrt(1.0 + g);
            nxx[p] = f * uxx[p];
            nxy[p] = f * uxy[p];
            nyy[p] = f * uyy[p];
        }
    }

    /* G_rho smoothing of the three fields (sampled Gaussian, mirror border)  */
    double *sm[3] = {nxx, nxy, nyy};
    int r = or_gauss_radius(rho);
    double *w0 = malloc(sizeof(double) * (2 * r + 1));
    double *w1 = malloc(sizeof(double) * (2 * r + 1));
    double *w2 = malloc(sizeof(double) * (2 * r + 1));
    or_gauss_kernels(rho, r, w0, w1, w2);
    double *tmp = malloc(sizeof(double) * np);
    for (int f = 0; f < 3; ++f) {
        double *F = sm[f];
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double acc = 0.0;
                for (int k = -r; k <= r; ++k)
                    acc += w0[k + r] * F[(size_t)y * w + or_mirror(x + k, w)];
                tmp[(size_t)y * w + x] = acc;
            }
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double acc = 0.0;
                for (int k = -r; k <= r; ++k)
                    acc += w0[k + r] * tmp[(size_t)or_mirror(y + k, h) * w + x];
                F[(size_t)y * w + x] = acc;
            }
    }

    for (size_t p = 0; p < np; ++p) {
        double a = nxx[p], b = nxy[p], d = nyy[p];
        /* principal-axis angle of the symmetric 2x2 matrix [[a b][b d]]     */
        double th = 0.5 * atan2(2.0 * b, a - d);
        double c1 = cos(th), s1 = sin(th);
        double nu1 = c1 * c1 * a + 2.0 * c1 * s1 * b + s1 * s1 * d;   /* e1' N e1 */
        double nu2 = s1 * s1 * a - 2.0 * c1 * s1 * b + c1 * c1 * d;   /* e2' N e2 */
        tensor[p] = cos(2.0 * th);
        tensor[np + p] = sin(2.0 * th);
        tensor[2 * np + p] = or_mu(nu1, lambda, mode);
        tensor[3 * np + p] = or_mu(nu2, lambda, mode);
        if (n_out) {
            n_out[p] = a;
            n_out[np + p] = b;
            n_out[2 * np + p] = d;
        }
    }
    free(tmp); free(w0); free(w1); free(w2);
    free(nxx); free(nxy); free(nyy);
    free(ux); free(uy); free(uxx); free(uxy); free(uyy);
}

/* The 4x4 matrix D_i = E M E^T of Sec. 3.4 acting on (xx, xy, yx, yy), built
 * from the eigentensors E_1..E_4 of Eq. 8 with mu3 = (mu1 + mu2)/2 and
 * mu4 = 0.  (c2, s2) = (cos 2theta, sin 2theta) of e1.                      */
void or_tensor_matrix(double c2, double s2, double mu1, double mu2, double *D)
{
    double th = 0.5 * atan2(s2, c2);
    double e1[2] = {cos(th), sin(th)};
    double e2[2] = {-sin(th), cos(th)};
    double E[4][4]; /* E[row = component (xx,xy,yx,yy)][col = k]              */
    const double is2 = 1.0 / sqrt(2.0);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            int row = 2 * i + j;
            E[row][0] = e1[i] * e1[j];
            E[row][1] = e2[i] * e2[j];
            E[row][2] = is2 * (e1[i] * e2[j] + e2[i] * e1[j]);
            E[row][3] = is2 * (e1[i] * e2[j] - e2[i] * e1[j]);
        }
    double mu[4] = {mu1, mu2, 0.5 * (mu1 + mu2), 0.0};
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k)
                acc += E[a][k] * mu[k] * E[b][k];
            D[4 * a + b] = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* The discrete operator P = L^T D L of Sec. 3.4 (Eq. 15-17) with the Hajiaboli stencils
 * (unit pixel size).  Natural boundary: a row of L exists only where its whole
 * stencil fits in the image; absent rows are zero (reading: per stencil, so
 * Lxx needs 1 <= x <= w-2, Lyy needs 1 <= y <= h-2, Lxy = Lyx needs both).
 * Periodic boundary (tests only): every row exists, indices wrap.
 * out = P u, computed literally: h = L u (4 components per pixel), T = D h per
 * pixel, then out = L^T T by scattering every row's stencil coefficients.   */
static double or_stencil_coef(int c, int dx, int dy)
{
    /* coefficient of u[x+dx, y+dy] in row (x, y) of component c            */
    switch (c) {
    case 0: /* xx */
        if (dy != 0) return 0.0;
        return dx == 0 ? -2.0 : 1.0;
    case 1: /* xy */
    case 2: /* yx */
        if (dx == 0 || dy == 0) return 0.0;
        return (dx == dy) ? 0.25 : -0.25;
    default: /* yy */
        if (dx != 0) return 0.0;
        return dy == 0 ? -2.0 : 1.0;
    }
}

static int or_row_valid(int c, int x, int y, int w, int h, int boundary)
{
    if (boundary == OR_PERIODIC)
        return 1;
    int okx = x >= 1 && x <= w - 2;
    int oky = y >= 1 && y <= h - 2;
    switch (c) {
    case 0: return okx;
    case 3: return oky;
    default: return okx && oky;
    }
}

static int or_wrap(int i, int n)
{
    int m = i % n;
    return m < 0 ? m + n : m;
}

void or_apply_P(const double *u, int w, int h, const double *tensor,
                int boundary, double *out)
{
    size_t np = (size_t)w * h;
    double *T = malloc(sizeof(double) * 4 * np);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double hv[4];
            for (int c = 0; c < 4; ++c) {
                hv[c] = 0.0;
                if (!or_row_valid(c, x, y, w, h, boundary))
                    continue;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        double co = or_stencil_coef(c, dx, dy);
                        if (co == 0.0)
                            continue;
                        int xx = boundary == OR_PERIODIC ? or_wrap(x + dx, w) : x + dx;
                        int yy = boundary == OR_PERIODIC ? or_wrap(y + dy, h) : y + dy;
                        hv[c] += co * u[(size_t)yy * w + xx];
                    }
            }
            double D[16];
            or_tensor_matrix(tensor[p], tensor[np + p], tensor[2 * np + p],
                             tensor[3 * np + p], D);
            for (int a = 0; a < 4; ++a) {
                double acc = 0.0;
                for (int b = 0; b < 4; ++b)
                    acc += D[4 * a + b] * hv[b];
                T[4 * p + a] = or_row_valid(a, x, y, w, h, boundary) ? acc : 0.0;
            }
        }
    }
    memset(out, 0, sizeof(double) * np);
    /* out = L^T T: row (x, y) of component c sends coef * T_c to each pixel
     * of its stencil (serial scatter: the transpose taken literally).      */
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            for (int c = 0; c < 4; ++c) {
                double t = T[4 * p + c];
                if (t == 0.0)
                    continue;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        double co = or_stencil_coef(c, dx, dy);
                        if (co == 0.0)
                            continue;
                        int xx = boundary == OR_PERIODIC ? or_wrap(x + dx, w) : x + dx;
                        int yy = boundary == OR_PERIODIC ? or_wrap(y + dy, h) : y + dy;
                        out[(size_t)yy * w + xx] += co * t;
                    }
            }
        }
    free(T);
}

/* ------------------------------------------------------------------------ */
/* FED step sizes (Sec. 3.5, Eq. 22-23).  n = ceil(-1/2 + 1/2 sqrt(1 + 12 T / (M tau_max)))
 * unless n_in > 0; tau_i = 3T / (2 M (n^2 + n) cos^2(pi (2i+1) / (4n+2))).
 * With n given, 3T/(M(n^2+n)) must not exceed tau_max (returns -1 if it does,
 * -2 on bad arguments).
 * Ordering (the paper uses the kappa-cycle rearrangement of the FED authors'
 * code, which is not reproduced in the paper).  Reading: the permutation
 * pi(i) = kappa * i mod n with gcd(kappa, n) = 1; kappa_in = 1 keeps the
 * natural order, kappa_in = 0 picks the kappa with the smallest rounding-error
 * growth bound
 *     A(kappa) = max_j  max_p |prod_{l < j} f_l(p)|  *  max_q |prod_{l >= j} f_l(q)|,
 * f_l(p) = 1 - tau_pi(l) p, p and q on 4096 points of [0, 34] (34 bounds
 * ||P||, Sec. 3.4, Eq. 19-20): the first factor bounds how far the state
 * before step j can grow, the second how far an error injected there can grow
 * by the end of the cycle.  Ties go to the smaller kappa.
 * tau_out[i] = tau_pi(i).
 * Returns 0; *n_out = n, *kappa_out = kappa used, *amp_out = A(kappa).      */
static double or_fed_amplification(const double *tau, int n, int kappa)
{
    const int NP = 4096;
    double worst = 0.0;
    for (int j = 0; j <= n; ++j) {
        double pre = 0.0, suf = 0.0;
        for (int ip = 0; ip < NP; ++ip) {
            double p = 34.0 * (double)ip / (double)(NP - 1);
            double a = 1.0, b = 1.0;
            for (int l = 0; l < j; ++l)
                a *= 1.0 - tau[(kappa * l) % n] * p;
            for (int l = j; l < n; ++l)
                b *= 1.0 - tau[(kappa * l) % n] * p;
            if (fabs(a) > pre) pre = fabs(a);
            if (fabs(b) > suf) suf = fabs(b);
        }
        if (pre * suf > worst)
            worst = pre * suf;
    }
    return worst;
}

static int or_gcd(int a, int b)
{
    while (b) {
        int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

int or_fed_taus(double T, int M, double tau_max, int n_in, int kappa_in,
                double *tau_out, int *n_out, int *kappa_out, double *amp_out)
{
    if (!(T > 0.0) || M <= 0 || !(tau_max > 0.0) || n_in < 0 || kappa_in < 0)
        return -2;
    int n = n_in;
    if (n == 0)
        n = (int)ceil(-0.5 + 0.5 * sqrt(1.0 + 12.0 * T / ((double)M * tau_max)));
    if (n < 1)
        n = 1;
    if (3.0 * T / ((double)M * ((double)n * n + n)) > tau_max * (1.0 + 1e-12))
        return -1;
    double *tau = malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) {
        double c = cos(OR_PI * (2.0 * i + 1.0) / (4.0 * n + 2.0));
        tau[i] = 3.0 * T / (2.0 * M * ((double)n * n + n) * c * c);
    }
    int kappa = kappa_in;
    double amp;
    if (kappa == 0) {
        double best = INFINITY;
        int arg = 1;
        for (int k = 1; k <= (n > 1 ? n - 1 : 1); ++k) {
            if (or_gcd(k, n) != 1)
                continue;
            double a = or_fed_amplification(tau, n, k);
            if (a < best) {
                best = a;
                arg = k;
            }
        }
        kappa = arg;
        amp = best;
    } else {
        if (n > 1 && or_gcd(kappa % n, n) != 1) {
            free(tau);
            return -2;
        }
        amp = or_fed_amplification(tau, n, kappa);
    }
    for (int i = 0; i < n; ++i)
        tau_out[i] = tau[(kappa * i) % n];
    free(tau);
    *n_out = n;
    if (kappa_out) *kappa_out = kappa;
    if (amp_out) *amp_out = amp;
    return 0;
}

/* One FED cycle (Sec. 3.5, Eq. 21): u <- (I - tau_i P) u for i = 0..n-1 with P frozen. */
void or_fed_cycle(double *u, int w, int h, const double *tensor,
                  const double *tau, int n, int boundary)
{
    size_t np = (size_t)w * h;
    double *Pu = malloc(sizeof(double) * np);
    for (int i = 0; i < n; ++i) {
        or_apply_P(u, w, h, tensor, boundary, Pu);
        for (size_t p = 0; p < np; ++p)
            u[p] -= tau[i] * Pu[p];
    }
    free(Pu);
}

/* The whole filter: sigma* once on the input (unless given), then M cycles of
 * (tensor from the current u at sigma*, one FED cycle).  u is filtered in
 * place.  sigma_idx_io: if sigma_given, read; else written.                 */
/* ------------------------------------------------------------------------ */
/* Crease extraction (Sec. 4, ridge and valley extraction): the zero contour
 * of d = det(g | Hg), g the gradient and H the Hessian of u_sigma, by marching
 * squares.  Readings (the paper names the method, not its discretisation):
 * derivatives of u_sigma at one scale sigma with the kernels of
 * or_gauss_kernels; cell (i, j) has the corners (i, j), (i+1, j), (i+1, j+1),
 * (i, j+1) (x to the right, y down), a corner is inside where d > 0, edge
 * crossings are linearly interpolated, a saddle cell (two diagonal corners
 * inside) is resolved by the mean of its corners (mean > 0: the inside corners
 * are connected); the zero set of d is a superset of the creases, and a cell's
 * segments are kept where the mean over its corners of the strongest Hessian
 * eigenvalue (the tie rule of or_select_scales) is negative (ridges) or
 * positive (valleys), or non-zero (both).                                   */
void or_crease_field(const double *u, int w, int h, double sigma, double *dfield, double *nu)
{
    size_t np = (size_t)w * h;
    double *ux = malloc(sizeof(double) * np), *uy = malloc(sizeof(double) * np);
    double *a = malloc(sizeof(double) * np), *b = malloc(sizeof(double) * np);
    double *d = malloc(sizeof(double) * np);
    or_derivatives(u, w, h, sigma, ux, uy, a, b, d);
    for (size_t p = 0; p < np; ++p) {
        double hgx = a[p] * ux[p] + b[p] * uy[p], hgy = b[p] * ux[p] + d[p] * uy[p];
        dfield[p] = ux[p] * hgy - uy[p] * hgx;
        double m = 0.5 * (a[p] + d[p]), r = hypot(0.5 * (a[p] - d[p]), b[p]);
        nu[p] = m > 0.0 ? m + r : m - r;
    }
    free(ux); free(uy); free(a); free(b); free(d);
}

/* Segments of the zero contour of d: 4 doubles (x0, y0, x1, y1) and a key
 * 2 * cell + k (cell = j * (w - 1) + i, k = 0 or 1) each, in key order; at most
 * max_segs written; returns the number found.                               */
int or_marching_squares(const double *d, const double *nu, int w, int h, int mode,
                        double *segs, int *keys, int max_segs)
{
    int n = 0;
    for (int j = 0; j + 1 < h; ++j)
        for (int i = 0; i + 1 < w; ++i) {
            double c[4] = {d[(size_t)j * w + i], d[(size_t)j * w + i + 1],
                           d[(size_t)(j + 1) * w + i + 1], d[(size_t)(j + 1) * w + i]};
            int cs = (c[0] > 0.0) | (c[1] > 0.0) << 1 | (c[2] > 0.0) << 2 | (c[3] > 0.0) << 3;
            if (cs == 0 || cs == 15)
                continue;
            double nm = 0.25 * (nu[(size_t)j * w + i] + nu[(size_t)j * w + i + 1] +
                                nu[(size_t)(j + 1) * w + i + 1] + nu[(size_t)(j + 1) * w + i]);
            if ((mode == OR_RIDGE && !(nm < 0.0)) || (mode == OR_VALLEY && !(nm > 0.0)) ||
                (mode == OR_BOTH && nm == 0.0))
                continue;
            /* crossing points on the edges top (0-1), right (1-2), bottom (3-2), left (0-3) */
            double ex[4], ey[4];
            ex[0] = i + c[0] / (c[0] - c[1]); ey[0] = j;
            ex[1] = i + 1;                    ey[1] = j + c[1] / (c[1] - c[2]);
            ex[2] = i + c[3] / (c[3] - c[2]); ey[2] = j + 1;
            ex[3] = i;                        ey[3] = j + c[0] / (c[0] - c[3]);
            int e0[2], e1[2], ns = 0;
            if (cs == 5 || cs == 10) { /* saddle: corners 0 and 2, or 1 and 3, inside */
                double mean = 0.25 * (c[0] + c[1] + c[2] + c[3]);
                int cut02 = (cs == 5) != (mean > 0.0); /* the segments cut off corners 0 and 2 */
                if (cut02) { e0[0] = 0; e1[0] = 3; e0[1] = 1; e1[1] = 2; }
                else       { e0[0] = 0; e1[0] = 1; e0[1] = 2; e1[1] = 3; }
                ns = 2;
            } else {
                static const int P0[4] = {0, 1, 3, 0}, P1[4] = {1, 2, 2, 3}; /* corners of edge e */
                int cross[4], nc = 0;
                for (int e = 0; e < 4; ++e)
                    if ((c[P0[e]] > 0.0) != (c[P1[e]] > 0.0))
                        cross[nc++] = e;
                e0[0] = cross[0];
                e1[0] = cross[1];
                ns = 1;
            }
            for (int k = 0; k < ns; ++k) {
                if (n < max_segs) {
                    segs[4 * n + 0] = ex[e0[k]]; segs[4 * n + 1] = ey[e0[k]];
                    segs[4 * n + 2] = ex[e1[k]]; segs[4 * n + 3] = ey[e1[k]];
                    keys[n] = 2 * (j * (w - 1) + i) + k;
                }
                ++n;
            }
        }
    return n;
}

/* ------------------------------------------------------------------------ */
/* The isotropic fourth-order comparator (IFOD, Eq. 2, the nonlinear
 * fourth-order diffusion of Lysaker et al. in the form of Didas et al.): the
 * diffusivity is the scalar g(||H(u)||_F^2) on every second derivative, i.e.
 * D = g I, which in this parameterisation is the tensor (1, 0, g, g) (both
 * eigenvalues g; the orientation is immaterial).  Readings: H is the Hessian
 * of u_sigma at the one regularisation scale sigma (1.0 in the paper's
 * experiments), ||H||_F^2 = u_xx^2 + 2 u_xy^2 + u_yy^2, and g has the
 * Perona-Malik form of Eq. 7, g(s) = 1 / (1 + s / lambda^2); no integration
 * scale and no gradient normalisation; g is rebuilt from u^k every cycle.    */
void or_build_tensor_ifod(const double *u, int w, int h, double sigma, double lambda,
                          double *tensor)
{
    size_t np = (size_t)w * h;
    double *a = malloc(sizeof(double) * np);
    double *b = malloc(sizeof(double) * np);
    double *d = malloc(sizeof(double) * np);
    or_derivatives(u, w, h, sigma, NULL, NULL, a, b, d);
    for (size_t p = 0; p < np; ++p) {
        double f2 = a[p] * a[p] + 2.0 * b[p] * b[p] + d[p] * d[p];
        double g = 1.0 / (1.0 + f2 / (lambda * lambda));
        tensor[p] = 1.0;
        tensor[np + p] = 0.0;
        tensor[2 * np + p] = g;
        tensor[3 * np + p] = g;
    }
    free(a); free(b); free(d);
}

void or_filter_ifod(double *u, int w, int h, double sigma, double lambda, int boundary,
                    const double *tau, int n, int M)
{
    size_t np = (size_t)w * h;
    double *tensor = malloc(sizeof(double) * 4 * np);
    for (int k = 0; k < M; ++k) {
        or_build_tensor_ifod(u, w, h, sigma, lambda, tensor);
        or_fed_cycle(u, w, h, tensor, tau, n, boundary);
    }
    free(tensor);
}

/* The whole filter: M cycles of (tensor build at the selected scales, FED
 * cycle).  The scale image is selected once on the input (the default
 * reading), or, with reselect, again on the current image u^k before every
 * cycle's tensor build; with postprocess every selection is followed by the
 * scale-image post-processing at threshold theta; a given scale image is used
 * for every cycle as it is.                                                  */
void or_filter(double *u, int w, int h, const double *sigmas, int n_sigma,
               double lambda, double rho, double beta, double c_in,
               double gamma, int mode, int grad_sq, int boundary,
               const double *tau, int n, int M, uint8_t *sigma_idx_io,
               int sigma_given, int reselect, int postprocess, double theta)
{
    size_t np = (size_t)w * h;
    double *tensor = malloc(sizeof(double) * 4 * np);
    double *vmax = postprocess ? malloc(sizeof(double) * np) : NULL;
    for (int k = 0; k < M; ++k) {
        if (!sigma_given && (k == 0 || reselect)) {
            or_select_scales(u, w, h, sigmas, n_sigma, mode, beta, c_in, gamma,
                             sigma_idx_io, vmax, NULL);
            if (postprocess)
                or_postprocess_scales(u, w, h, sigma_idx_io, vmax, sigmas, n_sigma, theta);
        }
        or_build_tensor(u, w, h, sigma_idx_io, sigmas, n_sigma, lambda, rho,
                        mode, grad_sq, tensor, NULL);
        or_fed_cycle(u, w, h, tensor, tau, n, boundary);
    }
    free(tensor);
    free(vmax);
}
