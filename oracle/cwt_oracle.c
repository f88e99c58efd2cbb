/*
 * cwt_oracle.c -- plain, slow, FP64 CPU oracle for the FFT-based continuous
 * wavelet transform (CWT) of multichannel EEG (arXiv 2506.07793).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA library: it works in the time
 * domain, with no FFT, so that it can check the GPU's frequency-domain path.
 *
 * What it computes (the result the paper's method reaches, written out):
 *
 *  1. The complex Morlet wavelet in the sigma-parametrisation of Eq. 3
 *     (Section "Fourier transformed formula").  With carrier F (Hz) and
 *     sigma = n_cycles, the time scale is a = sigma / (2 pi F) seconds and
 *     kappa = exp(-sigma^2 / 2).  The time-domain wavelet whose Fourier
 *     transform is Eq. 3 (up to constant factors that the unit-energy
 *     normalisation below removes) is
 *         psi(tau) = exp(-tau^2 / (2 a^2)) * (exp(i 2 pi F tau) - kappa).
 *     kappa makes the wavelet zero-mean (the Morlet correction term; with
 *     kappa = 0 it is the Gabor wavelet of Eq. 4).
 *
 *     The generalized Morse wavelet (GMW, Eq. 5) has no closed time-domain
 *     form: it is defined by its spectrum.  With the Heaviside step U in
 *     place of the printed sign() (the analytic GMW), peak frequency F and
 *     parameters beta, gamma:
 *         Psi(nu) = U(nu) alpha w^beta exp(-w^gamma),  w = w_p nu / F,
 *         w_p = (beta / gamma)^(1/gamma),  alpha = 2 (e gamma / beta)^(beta/gamma),
 *     so Psi peaks at nu = F with value 2.
 *
 *  2. The FFT path computes a CYCLIC convolution over the padded length N
 *     (Eq. 1 and Eq. 2: the inverse FFT of a product of spectra).  Sampling
 *     the analytic spectrum on N bins is the same as convolving cyclically
 *     with the N-periodised sampled wavelet
 *         p[m] = sum_{r in Z} psi((m + r N) / fs),   m = 0..N-1,
 *     (indices m > N/2 hold negative time).  The sum over r runs over every
 *     replica whose Gaussian envelope is not exactly zero in double.
 *     When the wavelet is not resolved by the N-point grid (its carrier lies
 *     below the first DFT bins, so the replicas cancel almost completely:
 *     the periodised energy is below 1e-6 of the replicas' own energy), that
 *     sum keeps only a few correct digits.  The same p is then reached from
 *     the other side of Poisson summation, as for the GMW below:
 *         p[m] = fs * IDFT_N(P)[m],  P[k] = sum_q Psi((k/N + q) fs),
 *     with Psi(nu) = a sqrt(2 pi) (exp(-sigma^2 (nu/F - 1)^2 / 2)
 *                                  - kappa exp(-sigma^2 (nu/F)^2 / 2))
 *     the continuous Fourier transform of psi (Eq. 3 in Hz with its
 *     absolute constant).  Each P[k] is a sum of positive-or-tiny terms
 *     evaluated to full relative precision, so nothing cancels.
 *     For the GMW the same periodised sampled wavelet is reached from its
 *     spectrum: by Poisson summation its DFT is proportional to
 *         P[k] = sum_{q >= 0} Psi((k/N + q) fs)
 *     (negative frequencies vanish under U), so p = IDFT_N(P), computed here
 *     by the O(N^2) definition of the inverse DFT (no FFT).
 *
 *  3. Each scale is normalised to unit discrete energy,
 *         pn[m] = p[m] / sqrt(sum_m |p[m]|^2),
 *     or, under MNE-python's convention (its Morlet wavelets are divided by
 *     sqrt(0.5) times their L2 norm), to sum_m |pn[m]|^2 = 2.
 *
 *  4. The signal x[0..n) is zero-padded to N and convolved cyclically:
 *         c[t] = sum_{m=0}^{n-1} x[m] * pn[(t - m) mod N],
 *     for the kept output positions t = 0, d, 2d, ... < n (decimation d).
 *     Power and phase are |c|^2 and atan2(Im c, Re c); the Python wrapper
 *     derives them from c.
 *
 * Everything is O(n * n_out) per (channel, scale) row, in double, with a
 * plain sequential sum.  Rows are independent, so they are spread over
 * POSIX threads; threading changes no arithmetic.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* Envelope exp(-u) is exactly 0.0 in double for u > 745.2, so replicas with
 * |tau| > a * sqrt(2 * 746) contribute nothing; 39 a is a safe bound. */
#define ORACLE_ENVELOPE_RADIUS 39.0

/* Step 1: the Morlet wavelet at time tau (seconds). */
static void morlet_psi(double tau, double F, double sigma, double *re, double *im)
{
    double a = sigma / (2.0 * ORACLE_PI * F);
    double env = exp(-(tau * tau) / (2.0 * a * a));
    double kappa = exp(-0.5 * sigma * sigma);
    double ph = 2.0 * ORACLE_PI * F * tau;
    *re = env * (cos(ph) - kappa);
    *im = env * sin(ph);
}

/* Gabor variant (kappa = 0, Eq. 4), kept for the pins that compare the two. */
static void gabor_psi(double tau, double F, double sigma, double *re, double *im)
{
    double a = sigma / (2.0 * ORACLE_PI * F);
    double env = exp(-(tau * tau) / (2.0 * a * a));
    double ph = 2.0 * ORACLE_PI * F * tau;
    *re = env * cos(ph);
    *im = env * sin(ph);
}

/* Step 1, GMW: Psi(nu) of Eq. 5 with U(nu), peak at nu = F (value 2). */
double oracle_gmw_spectrum(double nu, double F, double beta, double gamma)
{
    if (!(nu > 0.0))
        return 0.0;
    double wp = pow(beta / gamma, 1.0 / gamma);
    double w = wp * nu / F;
    double log_alpha = log(2.0) + (beta / gamma) * log(exp(1.0) * gamma / beta);
    /* alpha w^beta exp(-w^gamma), evaluated through its logarithm so that
     * neither w^beta nor alpha overflows on its own */
    return exp(log_alpha + beta * log(w) - pow(w, gamma));
}

/* p = scale * IDFT_N(P) (with the 1/N) of a real spectrum P, by the O(N^2)
 * definition: the N-th roots of unity exp(+2 pi i j / N) with the exponent
 * k m reduced mod N in integers, so that every angle is exact. */
static int idft_real_spectrum(const double *P, int N, double scale, double *p_re, double *p_im)
{
    double *c = (double *)malloc(sizeof(double) * (size_t)N);
    double *s = (double *)malloc(sizeof(double) * (size_t)N);
    if (!c || !s) {
        free(c);
        free(s);
        return -2;
    }
    for (int j = 0; j < N; ++j) {
        double ang = 2.0 * ORACLE_PI * (double)j / (double)N;
        c[j] = cos(ang);
        s[j] = sin(ang);
    }
    for (int m = 0; m < N; ++m) {
        double sre = 0.0, sim = 0.0;
        int j = 0; /* j = k m mod N, stepped by m */
        for (int k = 0; k < N; ++k) {
            sre += P[k] * c[j];
            sim += P[k] * s[j];
            j += m;
            if (j >= N)
                j -= N;
        }
        p_re[m] = scale * sre / (double)N;
        p_im[m] = scale * sim / (double)N;
    }
    free(c);
    free(s);
    return 0;
}

/* Step 2, GMW: P[k] = sum_{q >= 0} Psi((k/N + q) fs), then p = IDFT_N(P)
 * (with the 1/N).  Psi rises to its peak at F and falls after it, so the sum
 * over q stops at the first term past the peak that is exactly zero. */
static int gmw_periodised(double F, double beta, double gamma, double fs, int N, double *p_re,
                          double *p_im)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)N);
    if (!P)
        return -2;
    for (int k = 0; k < N; ++k) {
        double sum = 0.0;
        for (long q = 0;; ++q) {
            double nu = ((double)k / (double)N + (double)q) * fs;
            double term = oracle_gmw_spectrum(nu, F, beta, gamma);
            sum += term;
            if (nu > F && term == 0.0)
                break;
        }
        P[k] = sum;
    }
    int rc = idft_real_spectrum(P, N, 1.0, p_re, p_im);
    free(P);
    return rc;
}

/* Continuous Fourier transform of the Morlet (kind 0) or Gabor (kind 1)
 * wavelet of step 1 at nu Hz: int psi(tau) exp(-i 2 pi nu tau) dtau. */
double oracle_morlet_spectrum(int kind, double nu, double F, double sigma)
{
    double a = sigma / (2.0 * ORACLE_PI * F);
    double kappa = kind == 0 ? exp(-0.5 * sigma * sigma) : 0.0;
    double u = nu / F;
    double g = exp(-0.5 * sigma * sigma * (u - 1.0) * (u - 1.0)) -
               kappa * exp(-0.5 * sigma * sigma * u * u);
    return a * sqrt(2.0 * ORACLE_PI) * g;
}

/* Step 2 from the spectrum side for Morlet / Gabor (Poisson summation):
 * p = fs * IDFT_N(P), P[k] = sum_q Psi((k/N + q) fs) over every q whose
 * Gaussians are not exactly zero in double (both lie within 40 F / sigma of
 * nu = F and nu = 0). */
static int morlet_periodised_spectral(int kind, double F, double sigma, double fs, int N,
                                      double *p_re, double *p_im)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)N);
    if (!P)
        return -2;
    double reach = 40.0 * F / sigma;
    for (int k = 0; k < N; ++k) {
        double base = (double)k / (double)N;
        double q_lo = ceil(-reach / fs - base), q_hi = floor((F + reach) / fs - base);
        double sum = 0.0;
        for (double q = q_lo; q <= q_hi; q += 1.0)
            sum += oracle_morlet_spectrum(kind, (base + q) * fs, F, sigma);
        P[k] = sum;
    }
    int rc = idft_real_spectrum(P, N, fs, p_re, p_im);
    free(P);
    return rc;
}

/* Step 2: p[m] = sum_r psi((m + r N) / fs).  kind 0 = Morlet, 1 = Gabor
 * (sigma = n_cycles), 2 = GMW (sigma = beta; gamma used only here).
 * Returns 0, -1 on a bad argument, -2 on allocation failure. */
int oracle_periodised_wavelet(int kind, double F, double sigma, double gamma, double fs, int N,
                              double *p_re, double *p_im)
{
    if (N <= 0 || !(F > 0.0) || !(sigma > 0.0) || !(fs > 0.0) || kind < 0 || kind > 2)
        return -1;
    if (kind == 2) {
        if (!(gamma > 0.0))
            return -1;
        return gmw_periodised(F, sigma, gamma, fs, N, p_re, p_im);
    }
    double a = sigma / (2.0 * ORACLE_PI * F);
    double reach = ORACLE_ENVELOPE_RADIUS * a * fs; /* in samples */
    double e_raw = 0.0, e_per = 0.0; /* replicas' own energy, periodised energy */
    for (int m = 0; m < N; ++m) {
        double lo = ceil((-reach - (double)m) / (double)N);
        double hi = floor((reach - (double)m) / (double)N);
        double sre = 0.0, sim = 0.0;
        for (double r = lo; r <= hi; r += 1.0) {
            double tau = ((double)m + r * (double)N) / fs;
            double vre, vim;
            if (kind == 0)
                morlet_psi(tau, F, sigma, &vre, &vim);
            else
                gabor_psi(tau, F, sigma, &vre, &vim);
            sre += vre;
            sim += vim;
            e_raw += vre * vre + vim * vim;
        }
        p_re[m] = sre;
        p_im[m] = sim;
        e_per += sre * sre + sim * sim;
    }
    /* unresolved wavelet: the replicas cancel to below 1e-6 of their energy,
     * so the sum above has lost most of its digits; take the spectral side */
    if (e_per < 1e-6 * e_raw)
        return morlet_periodised_spectral(kind, F, sigma, fs, N, p_re, p_im);
    return 0;
}

/* Steps 2 + 3: the periodised wavelet of one scale with sum_m |w[m]|^2 = norm2
 * (1: unit energy; 2: MNE-python's convention). */
int oracle_wavelet_norm(int kind, double F, double sigma, double gamma, double fs, int N,
                        double norm2, double *w_re, double *w_im)
{
    int rc = oracle_periodised_wavelet(kind, F, sigma, gamma, fs, N, w_re, w_im);
    if (rc != 0)
        return rc;
    double e = 0.0;
    for (int m = 0; m < N; ++m)
        e += w_re[m] * w_re[m] + w_im[m] * w_im[m];
    if (!(e > 0.0) || !(norm2 > 0.0))
        return -1;
    double inv = sqrt(norm2 / e);
    for (int m = 0; m < N; ++m) {
        w_re[m] *= inv;
        w_im[m] *= inv;
    }
    return 0;
}

/* Steps 2 + 3 with unit energy. */
int oracle_wavelet(int kind, double F, double sigma, double gamma, double fs, int N, double *w_re,
                   double *w_im)
{
    return oracle_wavelet_norm(kind, F, sigma, gamma, fs, N, 1.0, w_re, w_im);
}

/* ------------------------------------------------------------------------ */
/* Step 4: direct cyclic convolution over selected (channel, scale) rows.   */

typedef struct {
    const double *x; /* [C][n] */
    int n, N, d, n_out;
    const double *wre, *wim; /* [S][N] unit-energy wavelets */
    const int *row_c, *row_s; /* rows to compute */
    int n_rows;
    double *out_re, *out_im; /* [n_rows][n_out] */
    int next;                /* next row to take (guarded by lock) */
    pthread_mutex_t lock;
} conv_job;

static void conv_row(const conv_job *J, int i)
{
    const double *x = J->x + (size_t)J->row_c[i] * (size_t)J->n;
    const double *wr = J->wre + (size_t)J->row_s[i] * (size_t)J->N;
    const double *wi = J->wim + (size_t)J->row_s[i] * (size_t)J->N;
    double *ore = J->out_re + (size_t)i * (size_t)J->n_out;
    double *oim = J->out_im + (size_t)i * (size_t)J->n_out;
    for (int o = 0; o < J->n_out; ++o) {
        int t = o * J->d;
        double sre = 0.0, sim = 0.0;
        for (int m = 0; m < J->n; ++m) {
            int idx = t - m;
            if (idx < 0)
                idx += J->N;
            sre += x[m] * wr[idx];
            sim += x[m] * wi[idx];
        }
        ore[o] = sre;
        oim[o] = sim;
    }
}

static void *conv_worker(void *arg)
{
    conv_job *J = (conv_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int i = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (i >= J->n_rows)
            break;
        conv_row(J, i);
    }
    return NULL;
}

/*
 * oracle_cwt_rows: CWT coefficients of the listed rows.
 *   x        [C][n] signal (double)
 *   N        cyclic length (>= n)
 *   fs       sampling rate (Hz)
 *   freqs, n_cycles [S]: carrier F_s and sigma_s of each scale (GMW: peak
 *            frequency F_s and beta_s)
 *   kind     0 = Morlet, 1 = Gabor, 2 = GMW (with gamma)
 *   d        decimation (>= 1); n_out = ceil(n / d)
 *   row_c, row_s [n_rows]: channel and scale index of each requested row
 *   norm2    sum_m |w[m]|^2 of every scale's wavelet (1 or 2, step 3)
 *   out_re, out_im [n_rows][n_out]
 *   n_threads worker threads (>= 1)
 * Returns 0 on success, -1 on a bad argument, -2 on allocation failure.
 */
int oracle_cwt_rows(const double *x, int C, int n, int N, double fs, const double *freqs,
                    const double *n_cycles, int S, int kind, double gamma, int d, const int *row_c,
                    const int *row_s, int n_rows, double norm2, double *out_re, double *out_im,
                    int n_threads)
{
    if (C <= 0 || n <= 0 || N < n || S <= 0 || d < 1 || n_rows < 0 || !(fs > 0.0))
        return -1;
    for (int i = 0; i < n_rows; ++i)
        if (row_c[i] < 0 || row_c[i] >= C || row_s[i] < 0 || row_s[i] >= S)
            return -1;
    if (n_threads < 1)
        n_threads = 1;
    double *wre = (double *)malloc(sizeof(double) * (size_t)S * (size_t)N);
    double *wim = (double *)malloc(sizeof(double) * (size_t)S * (size_t)N);
    if (!wre || !wim) {
        free(wre);
        free(wim);
        return -2;
    }
    int rc = 0;
    for (int s = 0; s < S && rc == 0; ++s)
        rc = oracle_wavelet_norm(kind, freqs[s], n_cycles[s], gamma, fs, N, norm2,
                                 wre + (size_t)s * N, wim + (size_t)s * N);
    if (rc == 0) {
        conv_job J;
        J.x = x;
        J.n = n;
        J.N = N;
        J.d = d;
        J.n_out = (n + d - 1) / d;
        J.wre = wre;
        J.wim = wim;
        J.row_c = row_c;
        J.row_s = row_s;
        J.n_rows = n_rows;
        J.out_re = out_re;
        J.out_im = out_im;
        J.next = 0;
        pthread_mutex_init(&J.lock, NULL);
        if (n_threads == 1) {
            conv_worker(&J);
        } else {
            pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
            int started = 0;
            if (th)
                for (; started < n_threads; ++started)
                    if (pthread_create(&th[started], NULL, conv_worker, &J) != 0)
                        break;
            conv_worker(&J); /* the caller's thread works too */
            for (int i = 0; i < started; ++i)
                pthread_join(th[i], NULL);
            free(th);
        }
        pthread_mutex_destroy(&J.lock);
    }
    free(wre);
    free(wim);
    return rc;
}

/* Brute-force O(N^2) DFT in double, sign -1 (forward) or +1 (inverse, no
 * 1/N).  Used only by the pins to cross-check indexing on tiny inputs. */
int oracle_dft(const double *in_re, const double *in_im, int N, int sign, double *out_re,
               double *out_im)
{
    if (N <= 0 || (sign != 1 && sign != -1))
        return -1;
    for (int k = 0; k < N; ++k) {
        double sre = 0.0, sim = 0.0;
        for (int m = 0; m < N; ++m) {
            /* angle reduced mod N in integers to keep it exact */
            long long km = ((long long)k * (long long)m) % (long long)N;
            double ang = (double)sign * 2.0 * ORACLE_PI * (double)km / (double)N;
            double c = cos(ang), s = sin(ang);
            sre += in_re[m] * c - in_im[m] * s;
            sim += in_re[m] * s + in_im[m] * c;
        }
        out_re[k] = sre;
        out_im[k] = sim;
    }
    return 0;
}
