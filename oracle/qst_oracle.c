/*
 * Plain FP64 CPU oracle of the pooled-chain pCN sampler for Bayesian quantum
 * state tomography (Nguyen, Law, Lukens, "Unorthodox parallelization for
 * Bayesian quantum state estimation", arXiv:2501.17334).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It is slow and
 * deliberately simple: complex<double> loops written in the order of the
 * paper's algorithms, with no blocking, fusion or reordering.  It shares no
 * code, header, table or constant with the CUDA implementation.
 *
 * Contents and the passages they follow:
 *   philox4x32_10     counter-based generator of Salmon, Moraes, Dror, Shaw,
 *                     "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
 *   normal draws      Box-Muller on the generator's uniforms (Algorithm 2: initial state and proposal noise).
 *   bures_rho         Algorithm 1 steps 2-6 (Householder QR, U = Q Lambda,
 *                     W = (U + I) G, rho = W W^dag / Tr W W^dag).
 *   hs_rho            the Hilbert-Schmidt prior, rho = G G^dag / Tr G G^dag (G as in
 *                     Algorithm 1; H unused), a prior the method admits in place of Bures.
 *   probabilities     p_kl = Tr(Lambda_kl rho) as a direct complex trace (Sec. II); with no
 *                     POVM arrays, Lambda_kl is the Pauli projector of setting k and outcome l,
 *                     each entry the product of the qubits' eigenprojector entries.
 *   loglik            log L = sum_kl c_kl log p_kl (Eq. likelihood).
 *   loglik_poisson    a non-multinomial likelihood (Sec. III: other likelihoods change only
 *                     the likelihood step of Algorithm 2): independent Poisson counts of mean
 *                     mu_k p_kl, mu_k the expected trials of setting k, whose elements need
 *                     not sum to the identity (lossy detectors).
 *   oracle_run        Algorithm 2 for chains [chain_begin, chain_begin+num_chains)
 *                     with step-size adaptation and thinning, pooled as in
 *                     Eq. BME2 / Step 6.
 *
 * Parity pins: see the oracle tests (Philox against cuRAND's own Philox4x32-10,
 * QR against LAPACK, Bures moments, the prior-sampling limit, a 1-qubit
 * posterior by quadrature, hand-computed likelihoods).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4.2 "Philox")              */
/* ------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* One bijection of the 128-bit counter under the 64-bit key: 10 rounds of the
 * S-box  (L0,R0,L1,R1) -> (hi(M1 R1) ^ L0 ^ k0, lo(M1 R1), hi(M0 R0) ^ L1 ^ k1, lo(M0 R0))
 * with R0 = word 0, R1 = word 2, L0 = word 1, L1 = word 3 and the Weyl key schedule. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream layout shared by contract (not by code) with the GPU path:
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (block b, step j, global chain id, stream tag)
 *   tag 0: the initial state y^0, tag 1: the proposal noise eta, tag 2: alpha. */
enum { TAG_INIT = 0, TAG_PROPOSAL = 1, TAG_ALPHA = 2 };

static void draw_block(uint64_t seed, uint32_t block, uint32_t step, uint32_t chain, uint32_t tag,
                       uint32_t out[4])
{
    uint32_t ctr[4] = {block, step, chain, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

/* Open-interval uniform from the top 23 bits: (2m+1) 2^-24, exact in float and double. */
static double uniform01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* n standard normals (n a multiple of 4): block b gives entries 4b..4b+3 by
 * Box-Muller on the uniform pairs (u0,u1) and (u2,u3):
 *   z = sqrt(-2 ln u_a) * (cos 2 pi u_b, sin 2 pi u_b). */
void oracle_normals(uint64_t seed, uint32_t step, uint32_t chain, uint32_t tag, int64_t n, double *z)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t b = 0; 4 * b < n; ++b) {
        uint32_t w[4];
        draw_block(seed, (uint32_t)b, step, chain, tag, w);
        for (int pair = 0; pair < 2; ++pair) {
            double ua = uniform01(w[2 * pair]);
            double ub = uniform01(w[2 * pair + 1]);
            double r = sqrt(-2.0 * log(ua));
            z[4 * b + 2 * pair] = r * cos(two_pi * ub);
            z[4 * b + 2 * pair + 1] = r * sin(two_pi * ub);
        }
    }
}

/* alpha ~ U(0,1) for step j of a chain (Algorithm 2, accept test): word 0 of block 0. */
double oracle_alpha(uint64_t seed, uint32_t step, uint32_t chain)
{
    uint32_t w[4];
    draw_block(seed, 0u, step, chain, TAG_ALPHA, w);
    return uniform01(w[0]);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: x in R^{4D^2} -> rho                                    */
/* ------------------------------------------------------------------ */

/* Householder QR of the D x D complex matrix H (column-major, H[a + D*b]).
 * Returns the unitary factor with its phases fixed, U = Q Lambda with
 * Lambda = diag(r_ii / |r_ii|) (Algorithm 1 steps 4-5), and the diagonal of R
 * before the fix.  Textbook complex Householder: for column k, the reflector
 * I - 2 v v^dag maps x = H[k:,k] to alpha e_1 with alpha = -e^{i arg x_0} |x|. */
void oracle_qr_unitary(int D, const cplx *H, cplx *U, cplx *rdiag)
{
    cplx *A = malloc(sizeof(cplx) * D * D);
    cplx *V = calloc((size_t)D * D, sizeof(cplx)); /* reflector k in column k, rows k.. */
    memcpy(A, H, sizeof(cplx) * D * D);
    for (int k = 0; k < D; ++k) {
        double xnorm = 0.0;
        for (int i = k; i < D; ++i) xnorm += creal(A[i + D * k] * conj(A[i + D * k]));
        xnorm = sqrt(xnorm);
        cplx x0 = A[k + D * k];
        cplx phase = (cabs(x0) > 0.0) ? x0 / cabs(x0) : 1.0;
        cplx alpha = -phase * xnorm;
        for (int i = k; i < D; ++i) V[i + D * k] = A[i + D * k];
        V[k + D * k] -= alpha;
        double vnorm = 0.0;
        for (int i = k; i < D; ++i) vnorm += creal(V[i + D * k] * conj(V[i + D * k]));
        vnorm = sqrt(vnorm);
        if (vnorm > 0.0) {
            for (int i = k; i < D; ++i) V[i + D * k] /= vnorm;
            for (int j = k; j < D; ++j) {
                cplx s = 0.0;
                for (int i = k; i < D; ++i) s += conj(V[i + D * k]) * A[i + D * j];
                for (int i = k; i < D; ++i) A[i + D * j] -= 2.0 * V[i + D * k] * s;
            }
        }
        rdiag[k] = A[k + D * k];
    }
    /* Q = H_0 H_1 ... H_{D-1} applied to the identity, last reflector first. */
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) U[i + D * j] = (i == j) ? 1.0 : 0.0;
    for (int k = D - 1; k >= 0; --k) {
        for (int j = 0; j < D; ++j) {
            cplx s = 0.0;
            for (int i = k; i < D; ++i) s += conj(V[i + D * k]) * U[i + D * j];
            for (int i = k; i < D; ++i) U[i + D * j] -= 2.0 * V[i + D * k] * s;
        }
    }
    /* U = Q Lambda: scale column k by r_kk / |r_kk| (Mezzadri's phase fix). */
    for (int k = 0; k < D; ++k) {
        cplx lam = (cabs(rdiag[k]) > 0.0) ? rdiag[k] / cabs(rdiag[k]) : 1.0;
        for (int i = 0; i < D; ++i) U[i + D * k] *= lam;
    }
    free(A);
    free(V);
}

/* Algorithm 1 steps 2-6.  x has 4 D^2 entries; the D x D blocks are filled
 * column-major (MATLAB reshape):  G[a,b] = x[a + D b] + i x[D^2 + a + D b],
 * H[a,b] = x[2 D^2 + a + D b] + i x[3 D^2 + a + D b].  rho is row-major
 * rho[a*D + b] = <a|rho|b>. */
void oracle_bures_rho(int D, const double *x, cplx *rho)
{
    const int d2 = D * D;
    cplx *G = malloc(sizeof(cplx) * d2);
    cplx *H = malloc(sizeof(cplx) * d2);
    cplx *U = malloc(sizeof(cplx) * d2);
    cplx *W = malloc(sizeof(cplx) * d2);
    cplx *rd = malloc(sizeof(cplx) * D);
    for (int e = 0; e < d2; ++e) {
        G[e] = x[e] + I * x[d2 + e];
        H[e] = x[2 * d2 + e] + I * x[3 * d2 + e];
    }
    oracle_qr_unitary(D, H, U, rd);
    /* W = (U + I_D) G   (the identity is D x D: U is D x D) */
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            cplx s = 0.0;
            for (int k = 0; k < D; ++k) {
                cplx uk = U[a + D * k] + ((a == k) ? 1.0 : 0.0);
                s += uk * G[k + D * b];
            }
            W[a + D * b] = s;
        }
    /* rho = W W^dag / Tr(W W^dag) */
    double tr = 0.0;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            cplx s = 0.0;
            for (int j = 0; j < D; ++j) s += W[a + D * j] * conj(W[b + D * j]);
            rho[a * D + b] = s;
            if (a == b) tr += creal(s);
        }
    for (int e = 0; e < d2; ++e) rho[e] /= tr;
    free(G); free(H); free(U); free(W); free(rd);
}

/* The Hilbert-Schmidt (Ginibre) prior: rho = G G^dag / Tr(G G^dag), G from the first 2 D^2
 * entries of x exactly as in Algorithm 1. */
void oracle_hs_rho(int D, const double *x, cplx *rho)
{
    const int d2 = D * D;
    double tr = 0.0;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            cplx s = 0.0;
            for (int j = 0; j < D; ++j) s += (x[a + D * j] + I * x[d2 + a + D * j]) * conj(x[b + D * j] + I * x[d2 + b + D * j]);
            rho[a * D + b] = s;
            if (a == b) tr += creal(s);
        }
    for (int e = 0; e < d2; ++e) rho[e] /= tr;
}

/* rho(x) under the prior: 0 Bures (Algorithm 1), 1 Hilbert-Schmidt. */
static void rho_of_x(int D, int prior, const double *x, cplx *rho)
{
    if (prior == 1) oracle_hs_rho(D, x, rho);
    else oracle_bures_rho(D, x, rho);
}

/* ------------------------------------------------------------------ */
/* Likelihood (Sec. III Step 4, Eq. likelihood)                          */
/* ------------------------------------------------------------------ */

/* Entry (i, j) of the single-qubit eigenprojector of setting s (0 X, 1 Y, 2 Z) with outcome b
 * (0: eigenvalue +1): (1 + X)/2, (1 - X)/2, (1 + Y)/2, (1 - Y)/2, |0><0|, |1><1| (Sec. II). */
static cplx pauli_entry(int s, int b, int i, int j)
{
    const double sg = b ? -1.0 : 1.0;
    if (s == 0) return (i == j) ? 0.5 : 0.5 * sg;                          /* X = [[0, 1], [1, 0]] */
    if (s == 1) return (i == j) ? 0.5 : (i == 0 ? -0.5 * I * sg : 0.5 * I * sg);   /* Y = [[0, -i], [i, 0]] */
    return (i == b && j == b) ? 1.0 : 0.0;
}

/* Lambda_kl[a, b] of Q qubits: setting k = sum_q s_q 3^(Q-1-q), outcome l = sum_q b_q 2^(Q-1-q),
 * row a and column b split into qubit bits the same way (qubit 0 most significant). */
static cplx pauli_projector_entry(int Q, int k, int l, int a, int b)
{
    cplx v = 1.0;
    for (int q = Q - 1; q >= 0; --q) {   /* qubit q is digit Q-1-q from the right */
        const int s = k % 3, o = l & 1, i = a & 1, j = b & 1;
        k /= 3; l >>= 1; a >>= 1; b >>= 1;
        v *= pauli_entry(s, o, i, j);
        if (v == 0.0) return 0.0;
    }
    return v;
}

/* p_kl = Re Tr(Lambda_kl rho) = Re sum_{a,b} Lambda[a,b] rho[b,a]; Lambda is row-major [KD][D][D],
 * or, with povm_re == NULL, the Pauli projector of pauli_projector_entry (KD = 6^Q). */
void oracle_probabilities(int D, int KD, const double *povm_re, const double *povm_im, const cplx *rho,
                          double *p)
{
    if (!povm_re) {
        int Q = 0;
        while ((1 << Q) < D) ++Q;
        for (int m = 0; m < KD; ++m) {
            cplx s = 0.0;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) {
                    const cplx lam = pauli_projector_entry(Q, m / D, m % D, a, b);
                    if (lam != 0.0) s += lam * rho[b * D + a];
                }
            p[m] = creal(s);
        }
        return;
    }
    for (int m = 0; m < KD; ++m) {
        const double *lr = povm_re + (size_t)m * D * D;
        const double *li = povm_im + (size_t)m * D * D;
        cplx s = 0.0;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) s += (lr[a * D + b] + I * li[a * D + b]) * rho[b * D + a];
        p[m] = creal(s);
    }
}

/* log L = sum over c_kl > 0 of c_kl log p_kl; a counted outcome with p <= 0 gives -inf
 * (0 log 0 is taken as 0: outcomes never observed contribute nothing). */
double oracle_loglik(int KD, const int32_t *counts, const double *p)
{
    double s = 0.0;
    for (int m = 0; m < KD; ++m) {
        if (counts[m] == 0) continue;
        if (!(p[m] > 0.0)) return -INFINITY;
        s += (double)counts[m] * log(p[m]);
    }
    return s;
}

/* Poisson counts c_kl of mean mu_k p_kl (k = m / D the setting of element m):
 * log L = sum_kl [c_kl log(mu_k p_kl) - mu_k p_kl], without the data-only - log c_kl! (the
 * multinomial form above leaves out its coefficient likewise).  A counted outcome with
 * p <= 0 gives -inf; an outcome never observed contributes - mu_k p_kl only. */
double oracle_loglik_poisson(int D, int KD, const int32_t *counts, const double *mu, const double *p)
{
    double s = 0.0;
    for (int m = 0; m < KD; ++m) {
        const double lambda = mu[m / D] * p[m];
        if (counts[m] > 0) {
            if (!(p[m] > 0.0)) return -INFINITY;
            s += (double)counts[m] * log(lambda);
        }
        s -= lambda;
    }
    return s;
}

/* the likelihood of a problem: 0 multinomial (Eq. likelihood), 1 Poisson (mu required) */
static double loglik_model(int D, int KD, int likelihood, const int32_t *counts, const double *mu, const double *p)
{
    return likelihood == 1 ? oracle_loglik_poisson(D, KD, counts, mu, p) : oracle_loglik(KD, counts, p);
}

/* rho(x) followed by its log-likelihood, for one latent vector. */
double oracle_loglik_of_x(int D, int prior, int likelihood, const double *mu, int KD, const double *povm_re,
                          const double *povm_im, const int32_t *counts, const double *x, double *rho_re,
                          double *rho_im, double *p_out)
{
    cplx *rho = malloc(sizeof(cplx) * D * D);
    double *p = malloc(sizeof(double) * KD);
    rho_of_x(D, prior, x, rho);
    oracle_probabilities(D, KD, povm_re, povm_im, rho, p);
    double ll = loglik_model(D, KD, likelihood, counts, mu, p);
    if (rho_re)
        for (int e = 0; e < D * D; ++e) { rho_re[e] = creal(rho[e]); rho_im[e] = cimag(rho[e]); }
    if (p_out) memcpy(p_out, p, sizeof(double) * KD);
    free(rho);
    free(p);
    return ll;
}

/* Batched helper: rows of x [n][4D^2] -> rho, p, logL (each output optional). */
void oracle_evaluate_batch(int D, int prior, int likelihood, const double *mu, int KD, const double *povm_re,
                           const double *povm_im, const int32_t *counts, int64_t n, const double *x, double *rho_re,
                           double *rho_im, double *p, double *logl)
{
    const int64_t nx = 4 * (int64_t)D * D, d2 = (int64_t)D * D;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double ll = oracle_loglik_of_x(D, prior, likelihood, mu, KD, povm_re, povm_im, counts, x + i * nx,
                                       rho_re ? rho_re + i * d2 : NULL, rho_im ? rho_im + i * d2 : NULL,
                                       p ? p + i * KD : NULL);
        if (logl) logl[i] = ll;
    }
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 over a range of chains, pooled as in Eq. BME2            */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t D;               /* Hilbert-space dimension 2^Q */
    int32_t KD;              /* number of POVM elements */
    const double *povm_re;   /* [KD][D][D] row-major */
    const double *povm_im;
    const int32_t *counts;   /* [KD] */
    uint64_t seed;
    int64_t chain_begin;     /* global id of the first chain */
    int64_t num_chains;
    int64_t num_steps;       /* steps j = 1..num_steps */
    double beta0;            /* initial beta (Algorithm 2, initialisation) */
    int32_t adapt_interval;  /* M_A; 0 = fixed beta */
    double acc_lo, acc_hi;   /* adaptation window [0.2, 0.6] */
    double adapt_factor;     /* 1.1 */
    double beta_max;         /* clamp keeping sqrt(1 - beta^2) real */
    int32_t thin;            /* T */
    int32_t burn_in;         /* pool only steps j > burn_in */
    int32_t trace_steps;     /* record the first trace_steps steps of every chain */
    int32_t traj_chains;     /* store the pooled trajectory of the first traj_chains chains */
    int32_t traj_capacity;   /* ... up to this many kept samples each */
    int32_t prior;           /* 0 Bures (Algorithm 1), 1 Hilbert-Schmidt */
    int32_t likelihood;      /* 0 multinomial (Eq. likelihood), 1 Poisson */
    const double *mu;        /* [KD / D] expected trials per setting (Poisson) */
} oracle_cfg;

typedef struct {
    double *pool_re, *pool_im;   /* [D*D] row-major sums over chains and kept steps */
    int64_t *num_pooled;         /* [1] number of pooled samples (chains x kept steps) */
    double *chain_pool_re;       /* optional [num_chains][D*D] per-chain sums */
    double *chain_pool_im;
    double *final_y;             /* optional [num_chains][4D^2] */
    double *final_logl;          /* optional [num_chains] */
    double *final_beta;          /* optional [num_chains] */
    int64_t *accepts;            /* optional [num_chains] accepted proposals */
    uint8_t *trace_accept;       /* optional [num_chains][trace_steps] */
    double *trace_logl_prop;     /* optional [num_chains][trace_steps] */
    double *trace_log_alpha;     /* optional [num_chains][trace_steps] */
    double *trace_logl_cur;      /* optional [num_chains][trace_steps] log L before the step */
    double *traj_re, *traj_im;   /* optional [traj_chains][traj_capacity][D*D] */
} oracle_out;

static void run_one_chain(const oracle_cfg *cfg, int64_t r, const oracle_out *out, double *pool_re_r,
                          double *pool_im_r, int64_t *kept_r)
{
    const int D = cfg->D, KD = cfg->KD, d2 = D * D, nx = 4 * D * D;
    const uint32_t chain = (uint32_t)(cfg->chain_begin + r);
    double *y = malloc(sizeof(double) * nx);
    double *yp = malloc(sizeof(double) * nx);
    double *eta = malloc(sizeof(double) * nx);
    double *p = malloc(sizeof(double) * KD);
    cplx *rho = malloc(sizeof(cplx) * d2);
    cplx *rhop = malloc(sizeof(cplx) * d2);

    /* initialisation: A = 0, beta = beta0, y^0 ~ N(0, I) */
    int64_t A = 0, acc_total = 0, kept = 0;
    double beta = cfg->beta0;
    oracle_normals(cfg->seed, 0u, chain, TAG_INIT, nx, y);
    rho_of_x(D, cfg->prior, y, rho);
    oracle_probabilities(D, KD, cfg->povm_re, cfg->povm_im, rho, p);
    double logl = loglik_model(D, KD, cfg->likelihood, cfg->counts, cfg->mu, p);

    for (int64_t j = 1; j <= cfg->num_steps; ++j) {
        /* proposal: eta ~ N(0, I), y' = sqrt(1 - beta^2) y + beta eta */
        oracle_normals(cfg->seed, (uint32_t)j, chain, TAG_PROPOSAL, nx, eta);
        double a = sqrt(1.0 - beta * beta);
        for (int e = 0; e < nx; ++e) yp[e] = a * y[e] + beta * eta[e];
        /* likelihood: rho(y') and L(y'); rho(y^{j-1}) and L(y^{j-1}) are kept from the last accept */
        rho_of_x(D, cfg->prior, yp, rhop);
        oracle_probabilities(D, KD, cfg->povm_re, cfg->povm_im, rhop, p);
        double loglp = loglik_model(D, KD, cfg->likelihood, cfg->counts, cfg->mu, p);
        /* accept test: alpha ~ U(0,1); accept iff log alpha < log L(y') - log L(y) */
        double log_alpha = log(oracle_alpha(cfg->seed, (uint32_t)j, chain));
        int accept = log_alpha < loglp - logl;
        if (cfg->trace_steps > 0 && j <= cfg->trace_steps) {
            int64_t t = r * cfg->trace_steps + (j - 1);
            if (out->trace_accept) out->trace_accept[t] = (uint8_t)accept;
            if (out->trace_logl_prop) out->trace_logl_prop[t] = loglp;
            if (out->trace_log_alpha) out->trace_log_alpha[t] = log_alpha;
            if (out->trace_logl_cur) out->trace_logl_cur[t] = logl;
        }
        if (accept) {
            memcpy(y, yp, sizeof(double) * nx);
            memcpy(rho, rhop, sizeof(cplx) * d2);
            logl = loglp;
            A += 1;
            acc_total += 1;
        }
        /* adaptation: every M_A steps rescale beta to keep A/M_A in [lo, hi], then reset A */
        if (cfg->adapt_interval > 0 && j % cfg->adapt_interval == 0) {
            double rate = (double)A / (double)cfg->adapt_interval;
            if (rate > cfg->acc_hi) beta = cfg->adapt_factor * beta;
            if (rate < cfg->acc_lo) beta = beta / cfg->adapt_factor;
            if (beta > cfg->beta_max) beta = cfg->beta_max;
            A = 0;
        }
        /* thinning and pooling (Eq. BME2): keep the current state every T steps and pool it */
        if (j % cfg->thin == 0 && j > cfg->burn_in) {
            for (int e = 0; e < d2; ++e) {
                pool_re_r[e] += creal(rho[e]);
                pool_im_r[e] += cimag(rho[e]);
            }
            if (r < cfg->traj_chains && kept < cfg->traj_capacity && out->traj_re) {
                int64_t base = ((int64_t)r * cfg->traj_capacity + kept) * d2;
                for (int e = 0; e < d2; ++e) {
                    out->traj_re[base + e] = creal(rho[e]);
                    out->traj_im[base + e] = cimag(rho[e]);
                }
            }
            kept += 1;
        }
    }
    if (out->final_y) memcpy(out->final_y + r * nx, y, sizeof(double) * nx);
    if (out->final_logl) out->final_logl[r] = logl;
    if (out->final_beta) out->final_beta[r] = beta;
    if (out->accepts) out->accepts[r] = acc_total;
    *kept_r = kept;
    free(y); free(yp); free(eta); free(p); free(rho); free(rhop);
}

/* Runs every chain independently (they never communicate) and pools the kept
 * states of all chains: sum_r sum_n rho(x^{n,r}) and the sample count N R. */
int oracle_run(const oracle_cfg *cfg, const oracle_out *out)
{
    if (cfg->D < 1 || cfg->KD < 1 || cfg->num_chains < 0 || cfg->thin < 1) return 1;
    if (cfg->likelihood == 1 && !cfg->mu) return 1;
    const int d2 = cfg->D * cfg->D;
    const int64_t R = cfg->num_chains;
    double *pr = calloc((size_t)(R > 0 ? R : 1) * d2, sizeof(double));
    double *pi = calloc((size_t)(R > 0 ? R : 1) * d2, sizeof(double));
    int64_t *kept = calloc((size_t)(R > 0 ? R : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < R; ++r) run_one_chain(cfg, r, out, pr + r * d2, pi + r * d2, kept + r);
    /* fixed-order reduction over chains: independent of the thread count */
    int64_t total = 0;
    for (int e = 0; e < d2; ++e) { out->pool_re[e] = 0.0; out->pool_im[e] = 0.0; }
    for (int64_t r = 0; r < R; ++r) {
        for (int e = 0; e < d2; ++e) {
            out->pool_re[e] += pr[r * d2 + e];
            out->pool_im[e] += pi[r * d2 + e];
        }
        total += kept[r];
    }
    if (out->chain_pool_re)
        for (int64_t i = 0; i < R * d2; ++i) { out->chain_pool_re[i] = pr[i]; out->chain_pool_im[i] = pi[i]; }
    *out->num_pooled = total;
    free(pr); free(pi); free(kept);
    return 0;
}

/* Wrappers on split real/imaginary arrays for foreign callers. */
void oracle_qr_unitary_split(int D, const double *h_re, const double *h_im, double *u_re, double *u_im,
                             double *r_re, double *r_im)
{
    cplx *H = malloc(sizeof(cplx) * D * D), *U = malloc(sizeof(cplx) * D * D), *rd = malloc(sizeof(cplx) * D);
    for (int e = 0; e < D * D; ++e) H[e] = h_re[e] + I * h_im[e];
    oracle_qr_unitary(D, H, U, rd);
    for (int e = 0; e < D * D; ++e) { u_re[e] = creal(U[e]); u_im[e] = cimag(U[e]); }
    for (int k = 0; k < D; ++k) { r_re[k] = creal(rd[k]); r_im[k] = cimag(rd[k]); }
    free(H); free(U); free(rd);
}

void oracle_probabilities_split(int D, int KD, const double *povm_re, const double *povm_im,
                                const double *rho_re, const double *rho_im, double *p)
{
    cplx *rho = malloc(sizeof(cplx) * D * D);
    for (int e = 0; e < D * D; ++e) rho[e] = rho_re[e] + I * rho_im[e];
    oracle_probabilities(D, KD, povm_re, povm_im, rho, p);
    free(rho);
}

void oracle_philox_blocks(uint64_t seed, uint32_t step, uint32_t chain, uint32_t tag, uint32_t block0,
                          int64_t nblocks, uint32_t *out)
{
    for (int64_t b = 0; b < nblocks; ++b) draw_block(seed, block0 + (uint32_t)b, step, chain, tag, out + 4 * b);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
