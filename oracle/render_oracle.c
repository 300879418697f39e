/*
 * FP64 reference renderer for the equirectangular splatting path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link or call
 * this file; it exists so that tests, the smoke check and the CPU baseline of
 * the benchmark have an independent, slow, obviously correct answer.
 *
 * What it computes (per pixel, no tiles, every Gaussian evaluated):
 *   - the 2D kernel G_i(u) = exp(-q/2), q = d^T C_i d with d the offset of the
 *     pixel centre from the projected mean, azimuth offset wrapped into
 *     [-W/2, W/2)                                  (Sec. 3.2; Sec. 4.2 map)
 *   - alpha_i = min(0.99, sigma_i G_i), skipped when q > 2 ln 255 or
 *     alpha_i < 1/255 (3DGS cut-offs; the paper gives none)
 *   - survivors ordered front to back by receiver distance, ties by index
 *     (Sec. 4.2 compositing rule and Algorithm 1 IntersectGaussians/Sort)
 *   - z[k] = sum_i T_i alpha_i a_i exp(j(phi0_i - 2 pi f_k L_i / c)),
 *     T_i = prod_{j<i} (1 - alpha_j), stopping before the Gaussian that would
 *     take T below 1e-4                     (Sec. 4.2 compositing rule, with
 *     s_i/d_i folded into the amplitude a_i and the subcarrier entering as the
 *     delay phase of the path length L_i, Sec. 3.1 channel model)
 * and the analytic FP64 gradient of a real loss through those steps, given
 * dL/dz (as dL/dRe + j dL/dIm) for every rendered pixel and subcarrier.
 *
 * Built with -ffp-contract=off so that results do not depend on whether the
 * host compiler fuses multiply-adds.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C_LIGHT 299792458.0
#define ORC_PI 3.14159265358979323846

typedef struct {
    double depth;
    int idx;
    double alpha;   /* clamped opacity actually used */
    double g;       /* kernel value exp(-q/2) */
    double dx, dy;  /* wrapped pixel-centre offsets from the projected mean */
    int clamped;    /* sigma*g exceeded the 0.99 clamp */
} orc_hit;

typedef struct {
    double q_max, alpha_min, alpha_max, t_min;
} orc_cutoffs;

static int orc_cmp_hit(const void* pa, const void* pb) {
    const orc_hit* a = (const orc_hit*)pa;
    const orc_hit* b = (const orc_hit*)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Offset wrapped into [-W/2, W/2). */
static double orc_wrap(double d, int W) { return d - (double)W * floor(d / (double)W + 0.5); }

/* Collect, for pixel (x, y), every Gaussian whose alpha survives the cut-offs,
 * ordered by (depth, index).  Returns the count. */
static int orc_gather(int N, const double* px, const double* py, const double* cxx,
                      const double* cxy, const double* cyy, const double* depth,
                      const unsigned char* valid, const double* sigma, int W, int x, int y,
                      const orc_cutoffs* cut, orc_hit* hits) {
    const double ux = x + 0.5, uy = y + 0.5;
    int n = 0;
    for (int i = 0; i < N; ++i) {
        if (!valid[i]) continue;
        double dx = orc_wrap(ux - px[i], W);
        double dy = uy - py[i];
        double q = cxx[i] * dx * dx + 2.0 * cxy[i] * dx * dy + cyy[i] * dy * dy;
        if (q > cut->q_max) continue;
        double g = exp(-0.5 * q);
        double a = sigma[i] * g;
        int clamped = 0;
        if (a > cut->alpha_max) { a = cut->alpha_max; clamped = 1; }
        if (a < cut->alpha_min) continue;
        hits[n].depth = depth[i];
        hits[n].idx = i;
        hits[n].alpha = a;
        hits[n].g = g;
        hits[n].dx = dx;
        hits[n].dy = dy;
        hits[n].clamped = clamped;
        ++n;
    }
    qsort(hits, (size_t)n, sizeof(orc_hit), orc_cmp_hit);
    return n;
}

/* Number of leading survivors that are composited before termination, and the
 * transmittance left after them. */
static int orc_terminate(const orc_hit* hits, int n, double t_min, double* t_out) {
    double T = 1.0;
    int m = 0;
    for (; m < n; ++m) {
        double Tn = T * (1.0 - hits[m].alpha);
        if (Tn < t_min) break;
        T = Tn;
    }
    *t_out = T;
    return m;
}

static void orc_set_cutoffs(orc_cutoffs* c, int exact) {
    if (exact) {
        c->q_max = INFINITY;
        c->alpha_min = 0.0;
        c->alpha_max = 0.99;
        c->t_min = 0.0;
    } else {
        c->q_max = 2.0 * log(255.0);
        c->alpha_min = 1.0 / 255.0;
        c->alpha_max = 0.99;
        c->t_min = 1e-4;
    }
}

/*
 * Forward render of a list of pixels.
 *   N Gaussians, per-Gaussian FP64 arrays; valid[i] = 0 means culled.
 *   amp = a_i (amplitude including the 1/d attenuation), phi0 = phase offset,
 *   plen = L_i path length in metres.
 *   f0 = frequency of subcarrier 0 in Hz, df = spacing; f_k = f0 + k df.
 *   pix[p] = y*W + x for p < npix.
 * Outputs: z[p*K*2 + 2k + {0,1}], t_final[p], n_used[p], sig[p] (the last three may
 * be NULL).  sig is a signature of which Gaussians were composited in which
 * order (sum of (index + 1) * (position + 1)), so that finite-difference tests
 * can tell when a perturbation changed the composited set.
 */
int oracle_render_fwd(int N, const double* px, const double* py, const double* cxx,
                      const double* cxy, const double* cyy, const double* depth,
                      const unsigned char* valid, const double* sigma, const double* amp,
                      const double* phi0, const double* plen, int H, int W, int K, double f0,
                      double df, int exact, int npix, const int* pix, double* z,
                      double* t_final, int* n_used, unsigned long long* sig, int nthreads) {
    if (N < 0 || H <= 0 || W <= 0 || K <= 0 || npix < 0) return -1;
    orc_cutoffs cut;
    orc_set_cutoffs(&cut, exact);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int err = 0;
#pragma omp parallel
    {
        orc_hit* hits = (orc_hit*)malloc(sizeof(orc_hit) * (size_t)(N > 0 ? N : 1));
        if (!hits) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 16)
        for (int p = 0; p < npix; ++p) {
            if (!hits) continue;
            int x = pix[p] % W, y = pix[p] / W;
            int n = orc_gather(N, px, py, cxx, cxy, cyy, depth, valid, sigma, W, x, y, &cut, hits);
            double Tend;
            int m = orc_terminate(hits, n, cut.t_min, &Tend);
            double* zp = z + (size_t)p * K * 2;
            for (int k = 0; k < 2 * K; ++k) zp[k] = 0.0;
            double T = 1.0;
            for (int s = 0; s < m; ++s) {
                const orc_hit* h = &hits[s];
                int i = h->idx;
                double w = T * h->alpha;
                for (int k = 0; k < K; ++k) {
                    double fk = f0 + k * df;
                    double psi = phi0[i] - 2.0 * ORC_PI * fk * plen[i] / ORC_C_LIGHT;
                    zp[2 * k] += w * amp[i] * cos(psi);
                    zp[2 * k + 1] += w * amp[i] * sin(psi);
                }
                T = T * (1.0 - h->alpha);
            }
            if (t_final) t_final[p] = T;
            if (n_used) n_used[p] = m;
            if (sig) {
                unsigned long long acc = 0;
                for (int s = 0; s < m; ++s)
                    acc += (unsigned long long)(hits[s].idx + 1) * (unsigned long long)(s + 1);
                sig[p] = acc;
            }
        }
        free(hits);
    }
    return err;
}

/*
 * Analytic gradient.  gz[p*K*2 + 2k + {0,1}] = dL/dRe z, dL/dIm z.
 * grad is [N, 9], ACCUMULATED, columns:
 *   0 d p_x, 1 d p_y, 2 d c_xx, 3 d c_xy, 4 d c_yy, 5 d sigma, 6 d a, 7 d phi0, 8 d L
 * Derivation (hand-written, pinned by finite differences in the tests):
 *   with w_i = T_i alpha_i and Gc_i = sum_k conj(g_k) e^{j psi_ik},
 *   Fc_i = sum_k f_k conj(g_k) e^{j psi_ik}:
 *   dL/da_i     = w_i Re Gc_i
 *   dL/dphi0_i  = -w_i a_i Im Gc_i
 *   dL/dL_i     = (2 pi / c) w_i a_i Im Fc_i
 *   dL/dalpha_i = T_i a_i Re Gc_i - (1/(1-alpha_i)) sum_{m>i} w_m a_m Re Gc_m
 *   alpha = min(0.99, sigma g): dalpha/dsigma = g, dalpha/dg = sigma (0 if clamped)
 *   g = exp(-q/2), q = c_xx dx^2 + 2 c_xy dx dy + c_yy dy^2, dx = wrap(u_x - p_x).
 */
int oracle_render_bwd(int N, const double* px, const double* py, const double* cxx,
                      const double* cxy, const double* cyy, const double* depth,
                      const unsigned char* valid, const double* sigma, const double* amp,
                      const double* phi0, const double* plen, int H, int W, int K, double f0,
                      double df, int exact, int npix, const int* pix, const double* gz,
                      double* grad, int nthreads) {
    if (N < 0 || H <= 0 || W <= 0 || K <= 0 || npix < 0) return -1;
    orc_cutoffs cut;
    orc_set_cutoffs(&cut, exact);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    int nt = omp_get_max_threads();
#else
    int nt = 1;
#endif
    double* part = (double*)calloc((size_t)nt * (size_t)N * 9 + 1, sizeof(double));
    if (!part) return -2;
    int err = 0;
#pragma omp parallel
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        double* acc = part + (size_t)tid * N * 9;
        orc_hit* hits = (orc_hit*)malloc(sizeof(orc_hit) * (size_t)(N > 0 ? N : 1));
        double* ReG = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double* ImG = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double* ImF = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double* Ts = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        if (!hits || !ReG || !ImG || !ImF || !Ts) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(static)
        for (int p = 0; p < npix; ++p) {
            if (err) continue;
            int x = pix[p] % W, y = pix[p] / W;
            int n = orc_gather(N, px, py, cxx, cxy, cyy, depth, valid, sigma, W, x, y, &cut, hits);
            double Tend;
            int m = orc_terminate(hits, n, cut.t_min, &Tend);
            const double* g = gz + (size_t)p * K * 2;
            double T = 1.0;
            for (int s = 0; s < m; ++s) {
                int i = hits[s].idx;
                double re = 0.0, im = 0.0, imf = 0.0;
                for (int k = 0; k < K; ++k) {
                    double fk = f0 + k * df;
                    double psi = phi0[i] - 2.0 * ORC_PI * fk * plen[i] / ORC_C_LIGHT;
                    double c = cos(psi), sn = sin(psi);
                    /* conj(g) * e^{j psi} = (gr - j gi)(c + j sn) */
                    double pr = g[2 * k] * c + g[2 * k + 1] * sn;
                    double pi_ = g[2 * k] * sn - g[2 * k + 1] * c;
                    re += pr;
                    im += pi_;
                    imf += fk * pi_;
                }
                ReG[s] = re;
                ImG[s] = im;
                ImF[s] = imf;
                Ts[s] = T;
                T = T * (1.0 - hits[s].alpha);
            }
            double suffix = 0.0; /* sum_{m>s} w_m a_m Re Gc_m */
            for (int s = m - 1; s >= 0; --s) {
                const orc_hit* h = &hits[s];
                int i = h->idx;
                double w = Ts[s] * h->alpha;
                double* gi = acc + (size_t)i * 9;
                gi[6] += w * ReG[s];
                gi[7] += -w * amp[i] * ImG[s];
                gi[8] += (2.0 * ORC_PI / ORC_C_LIGHT) * w * amp[i] * ImF[s];
                double dalpha = Ts[s] * amp[i] * ReG[s] - suffix / (1.0 - h->alpha);
                suffix += w * amp[i] * ReG[s];
                if (h->clamped) continue;
                gi[5] += dalpha * h->g;
                double dq = dalpha * sigma[i] * h->g * (-0.5);
                double dx = h->dx, dy = h->dy;
                gi[0] += dq * (-(2.0 * cxx[i] * dx + 2.0 * cxy[i] * dy));
                gi[1] += dq * (-(2.0 * cxy[i] * dx + 2.0 * cyy[i] * dy));
                gi[2] += dq * dx * dx;
                gi[3] += dq * 2.0 * dx * dy;
                gi[4] += dq * dy * dy;
            }
        }
        free(hits);
        free(ReG);
        free(ImG);
        free(ImF);
        free(Ts);
    }
    if (!err) {
        for (int t = 0; t < nt; ++t) {
            const double* a = part + (size_t)t * N * 9;
            for (size_t j = 0; j < (size_t)N * 9; ++j) grad[j] += a[j];
        }
    }
    free(part);
    return err;
}
