// Host side of the C ABI declared in include/qst.h: validation, projector packing,
// workspace layout, the step loop, read-back, checkpointing and profiling.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/qst.h"
#include "qst_internal.cuh"

using namespace qst;

namespace {

thread_local std::string g_last_error;

qst_status fail(qst_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

qst_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(QST_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(QST_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define QST_CUDA(call, what)                      \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Packs Lambda (row-major [KD][D][D]) into P[(i,j)][m] with stride ld (see qst.h).
void pack_projectors(int D, int KD, const double *re, const double *im, double *P, int ld) {
    for (int m = 0; m < KD; ++m) {
        const double *lr = re + (size_t)m * D * D;
        const double *li = im + (size_t)m * D * D;
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                double v;
                if (i == j) v = lr[i * D + i];
                else if (i < j) v = 2.0 * lr[i * D + j];
                else v = 2.0 * li[i * D + j];
                P[(size_t)(i * D + j) * ld + m] = v;
            }
    }
}

// Is v a bf16 value up to FP64 round-off of its construction (relative 1e-12, the same
// tolerance as the completeness check)?  Then the bf16 value is used.
// operand kind of the tensor-core projection for a precision (TC_NONE: the plain FP32 form)
int tc_kind_of(int32_t precision) {
    switch (precision) {
        case QST_PREC_BF16X3: return TC_BF16X3;
        case QST_PREC_TF32: return TC_TF32;
        case QST_PREC_TF32X2: return TC_TF32X2;
        default: return TC_NONE;
    }
}

// v is exactly a TF32 value: an FP32 value whose 13 low mantissa bits are zero
bool tf32_exact(double v) {
    const float f = (float)v;
    if ((double)f != v) return false;
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return (u & 0x1FFFu) == 0u;
}

bool bf16_exact(double v) {
    const double r = (double)__bfloat162float(__float2bfloat16_rn((float)v));
    return std::fabs(r - v) <= 1e-12 * std::fabs(v);
}

// ------------------------------------------------------------------------------------------
// Per-problem host record and workspace layout
// ------------------------------------------------------------------------------------------
struct Layout {
    size_t P32, Ptc, cnt, invf, ptot, colw, pauli_wq, pauli_wc, pauli_perm, y, cur, rho_cur, rho_prop, rho_split, trace_prop, logl_cur, logl_part, beta, coef,
        acc_win,
        acc_total, pool, traj, trace_acc, trace_logl, red, acf, logl_eval, end;
};

struct HostProblem {
    ProblemView v{};
    int Q = 0, K = 0, KDmax = 0;
    int part_slots = 0;               // partial sums per chain the workspace holds (largest schedule)
    std::vector<int> group_choices;   // candidate ngroups values for the autotuner
    // QST_PREC_AUTO: the forms this problem's projection can take, and the tensor-core form's
    // column-group rule and candidates (kept while the structured Pauli form is in use)
    bool can_tc = false, can_pauli = false;
    int tc_groups_rule = 0;
    std::vector<int> tc_group_choices;
    double beta0 = 0.0;
    Layout off{};
    std::vector<float> P32;
    std::vector<__nv_bfloat16> Pbf;   // tensor-core B operand, BF16x3
    std::vector<float> Ptf;           // tensor-core B operand, TF32 forms
    std::vector<float> cnt, invf, ptot;
    std::vector<float4> pauli_wq;     // structured Pauli form: deviance weights per output pair
    std::vector<float2> pauli_wc;     // and counts
    std::vector<int32_t> pauli_perm;  // tree order -> setting-major projector index
    TcPlan *tc = nullptr;
};

struct Plan {
    std::vector<HostProblem> probs;
    size_t status_off = 0;  // device status word
    size_t step_off = 0;    // device StepState
    size_t bytes = 0;       // total workspace bytes
};

qst_status validate_cfg(const qst_sampler_cfg *cfg) {
    if (!cfg) return fail(QST_ERR_INVALID_ARG, "cfg is NULL");
    if (!(cfg->beta0 > 0.0) || !(cfg->beta_max <= 1.0) || !(cfg->beta0 <= cfg->beta_max))
        return fail(QST_ERR_INVALID_ARG, "need 0 < beta0 <= beta_max <= 1 (beta0=%g, beta_max=%g)", cfg->beta0,
                    cfg->beta_max);
    if (cfg->adapt_interval < 0) return fail(QST_ERR_INVALID_ARG, "adapt_interval must be >= 0");
    if (!(cfg->adapt_factor > 0.0)) return fail(QST_ERR_INVALID_ARG, "adapt_factor must be > 0");
    if (!(cfg->acc_lo <= cfg->acc_hi)) return fail(QST_ERR_INVALID_ARG, "need acc_lo <= acc_hi");
    if (cfg->thin < 1) return fail(QST_ERR_INVALID_ARG, "thin (T) must be >= 1");
    if (cfg->burn_in < 0) return fail(QST_ERR_INVALID_ARG, "burn_in must be >= 0");
    if (cfg->diag_chains < 0 || cfg->traj_capacity < 0 || cfg->acf_lmax < 0 || cfg->trace_steps < 0)
        return fail(QST_ERR_INVALID_ARG, "diagnostic sizes must be >= 0");
    if (cfg->precision != QST_PREC_FP32 && cfg->precision != QST_PREC_BF16X3 && cfg->precision != QST_PREC_TF32 &&
        cfg->precision != QST_PREC_TF32X2 && cfg->precision != QST_PREC_PAULI && cfg->precision != QST_PREC_AUTO)
        return fail(QST_ERR_INVALID_ARG, "unknown precision %d", cfg->precision);
    if (cfg->qr_passes < 1 || cfg->qr_passes > 4) return fail(QST_ERR_INVALID_ARG, "qr_passes must be 1, 2, 3 or 4");
    if (cfg->prior != QST_PRIOR_BURES && cfg->prior != QST_PRIOR_HS)
        return fail(QST_ERR_INVALID_ARG, "unknown prior %d", cfg->prior);
    if (cfg->use_graph != 0 && cfg->use_graph != 1) return fail(QST_ERR_INVALID_ARG, "use_graph must be 0 or 1");
    if (cfg->autotune != 0 && cfg->autotune != 1) return fail(QST_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (cfg->propose_threads != 0 && cfg->propose_threads != 32 && cfg->propose_threads != 64 &&
        cfg->propose_threads != 128)
        return fail(QST_ERR_INVALID_ARG, "propose_threads must be 0, 32, 64 or 128");
    return QST_OK;
}

// Upper bound on the POVM elements K D of one problem (2^20; six-qubit Pauli tomography has
// 46,656): keeps K D, K D D^2 and the padded sizes far from int and size_t limits.
constexpr int kMaxPovmElements = 1 << 20;

void pauli_povms(int Q, std::vector<double> &re, std::vector<double> &im);

// Qubits the forms cover: 1..5, and 6 for the structured Pauli form with the built-in POVMs
// (NULL arrays: as dense [K*D][D][D] arrays they would take 3 GB).
int max_qubits(const qst_sampler_cfg *cfg, bool builtin) {
    return (cfg->precision == QST_PREC_PAULI || cfg->precision == QST_PREC_AUTO) && builtin ? 6 : 5;
}

// The POVM arrays of d are the built-in Pauli set (to 1e-12).
bool povms_are_pauli(const qst_problem_desc &d) {
    if (d.num_povms != (int32_t)std::lround(std::pow(3.0, d.num_qubits))) return false;
    std::vector<double> pre, pim;
    pauli_povms(d.num_qubits, pre, pim);
    for (size_t e = 0; e < pre.size(); ++e)
        if (std::fabs(d.povm_re[e] - pre[e]) > 1e-12 || std::fabs(d.povm_im[e] - pim[e]) > 1e-12) return false;
    return true;
}

qst_status validate_problem(const qst_problem_desc &d, int idx, const qst_sampler_cfg *cfg) {
    const bool builtin = !d.povm_re && !d.povm_im;   // only the Pauli form keeps them unmaterialised
    if (d.num_qubits < 1 || d.num_qubits > max_qubits(cfg, builtin))
        return fail(QST_ERR_INVALID_ARG, "problem %d: num_qubits %d outside 1..%d", idx, d.num_qubits,
                    max_qubits(cfg, builtin));
    // bounded before any product with D is formed (K D and K D D^2 must not wrap)
    if (d.num_povms < 1 || d.num_povms > kMaxPovmElements >> d.num_qubits)
        return fail(QST_ERR_INVALID_ARG, "problem %d: num_povms must be in 1..2^20 / 2^Q", idx);
    if (!d.counts || (!builtin && (!d.povm_re || !d.povm_im)))
        return fail(QST_ERR_INVALID_ARG, "problem %d: NULL input", idx);
    if (tc_kind_of(cfg->precision) != TC_NONE && !tc_supported(tc_kind_of(cfg->precision), 1 << d.num_qubits))
        return fail(QST_ERR_INVALID_ARG, "problem %d: precision %d does not cover %d qubits (TF32: 1..4, TF32x2: 1..3)",
                    idx, cfg->precision, d.num_qubits);
    if (d.num_chains < 1) return fail(QST_ERR_INVALID_ARG, "problem %d: num_chains must be >= 1", idx);
    if (d.chain_offset < 0 || d.chain_offset + d.num_chains > (int64_t(1) << 32))
        return fail(QST_ERR_INVALID_ARG, "problem %d: chain ids must fit 32 bits", idx);
    if (!(d.beta0 >= 0.0) || d.beta0 > 1.0)
        return fail(QST_ERR_INVALID_ARG, "problem %d: beta0 %g outside [0, 1] (0 = the config's)", idx, d.beta0);
    if (d.beta0 > cfg->beta_max)
        return fail(QST_ERR_INVALID_ARG, "problem %d: beta0 %g above beta_max %g", idx, d.beta0, cfg->beta_max);
    const int D = 1 << d.num_qubits, KD = d.num_povms * D;
    for (int m = 0; m < KD; ++m)
        if (d.counts[m] < 0) return fail(QST_ERR_INVALID_ARG, "problem %d: negative count at %d", idx, m);
    if (d.likelihood != QST_LIKELIHOOD_MULTINOMIAL && d.likelihood != QST_LIKELIHOOD_POISSON)
        return fail(QST_ERR_INVALID_ARG, "problem %d: unknown likelihood %d", idx, d.likelihood);
    const bool poisson = d.likelihood == QST_LIKELIHOOD_POISSON;
    if (poisson) {
        if (!d.trials) return fail(QST_ERR_INVALID_ARG, "problem %d: the Poisson likelihood needs trials", idx);
        for (int k = 0; k < d.num_povms; ++k)
            if (!(d.trials[k] > 0.0) || !std::isfinite(d.trials[k]) || (double)(float)d.trials[k] != d.trials[k])
                return fail(QST_ERR_INVALID_ARG, "problem %d: trials[%d] must be > 0 and exact in FP32", idx, k);
    }
    if (builtin) {   // the built-in Pauli set (make_plan checked num_povms = 3^Q)
        if (cfg->precision != QST_PREC_PAULI && cfg->precision != QST_PREC_AUTO)
            return fail(QST_ERR_INVALID_ARG, "problem %d: NULL input", idx);
        return QST_OK;
    }
    // Hermitian elements, completeness per setting
    for (int m = 0; m < KD; ++m) {
        const double *re = d.povm_re + (size_t)m * D * D, *im = d.povm_im + (size_t)m * D * D;
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                if (!std::isfinite(re[i * D + j]) || !std::isfinite(im[i * D + j]))
                    return fail(QST_ERR_INVALID_ARG, "problem %d: non-finite POVM entry", idx);
                if (std::fabs(re[i * D + j] - re[j * D + i]) > 1e-12 || std::fabs(im[i * D + j] + im[j * D + i]) > 1e-12)
                    return fail(QST_ERR_INVALID_ARG, "problem %d: POVM element %d is not Hermitian", idx, m);
            }
    }
    for (int k = 0; k < d.num_povms; ++k)
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                double sr = 0.0, si = 0.0;
                for (int l = 0; l < D; ++l) {
                    sr += d.povm_re[((size_t)(k * D + l) * D + i) * D + j];
                    si += d.povm_im[((size_t)(k * D + l) * D + i) * D + j];
                    if (poisson && i == j && d.povm_re[((size_t)(k * D + l) * D + i) * D + j] < -1e-12)
                        return fail(QST_ERR_INVALID_ARG, "problem %d: element %d has a negative diagonal entry",
                                    idx, k * D + l);
                }
                if (poisson) {   // a sub-normalised setting: diagonal of the sum within [0, 1]
                    if (i == j && sr > 1.0 + 1e-12)
                        return fail(QST_ERR_INVALID_ARG, "problem %d: setting %d sums above the identity", idx, k);
                } else if (std::fabs(sr - (i == j ? 1.0 : 0.0)) > 1e-12 || std::fabs(si) > 1e-12) {
                    return fail(QST_ERR_INVALID_ARG, "problem %d: setting %d does not sum to the identity", idx, k);
                }
            }
    if (cfg->precision == QST_PREC_PAULI) {   // the structured form assumes the Pauli POVMs
        if (d.num_povms != (int32_t)std::lround(std::pow(3.0, d.num_qubits)))
            return fail(QST_ERR_INVALID_ARG, "problem %d: QST_PREC_PAULI needs the 3^Q Pauli settings", idx);
        std::vector<double> pre, pim;
        pauli_povms(d.num_qubits, pre, pim);
        for (size_t e = 0; e < pre.size(); ++e)
            if (std::fabs(d.povm_re[e] - pre[e]) > 1e-12 || std::fabs(d.povm_im[e] - pim[e]) > 1e-12)
                return fail(QST_ERR_INVALID_ARG, "problem %d: QST_PREC_PAULI needs the built-in Pauli POVMs", idx);
    }
    return QST_OK;
}

// The built-in Pauli POVMs of Q qubits, [3^Q * 2^Q][2^Q][2^Q] real and imaginary parts: setting
// k = sum_q s_q 3^(Q-1-q) (s = 0, 1, 2 for X, Y, Z), outcome l = sum_q b_q 2^(Q-1-q) (b = 0 for
// the +1 eigenvalue), qubit 0 the most significant Kronecker factor.  Every entry is 0 or
// +-2^-m (times 1 or i), exact in double.
void pauli_povms(int Q, std::vector<double> &re, std::vector<double> &im) {
    const int D = 1 << Q, K = (int)std::lround(std::pow(3.0, Q));
    // single-qubit eigenprojectors [setting][outcome][row][col] as (re, im)
    static const double pr[3][2][2][2] = {{{{0.5, 0.5}, {0.5, 0.5}}, {{0.5, -0.5}, {-0.5, 0.5}}},
                                          {{{0.5, 0.0}, {0.0, 0.5}}, {{0.5, 0.0}, {0.0, 0.5}}},
                                          {{{1.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {0.0, 1.0}}}};
    static const double pi[3][2][2][2] = {{{{0.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {0.0, 0.0}}},
                                          {{{0.0, -0.5}, {0.5, 0.0}}, {{0.0, 0.5}, {-0.5, 0.0}}},
                                          {{{0.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {0.0, 0.0}}}};
    re.assign((size_t)K * D * D * D, 0.0);
    im.assign((size_t)K * D * D * D, 0.0);
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < D; ++l)
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double ar = 1.0, ai = 0.0;   // product over qubits of the factors' (i_q, j_q) entries
                    for (int q = 0; q < Q; ++q) {
                        int kk = k;
                        for (int t = q + 1; t < Q; ++t) kk /= 3;
                        const int sq = kk % 3, bq = (l >> (Q - 1 - q)) & 1;
                        const int iq = (i >> (Q - 1 - q)) & 1, jq = (j >> (Q - 1 - q)) & 1;
                        const double fr = pr[sq][bq][iq][jq], fi = pi[sq][bq][iq][jq];
                        const double nr = ar * fr - ai * fi, ni = ar * fi + ai * fr;
                        ar = nr;
                        ai = ni;
                    }
                    const size_t e = (((size_t)(k * D + l) * D + i) * D + j);
                    re[e] = ar;
                    im[e] = ai;
                }
}

qst_status make_plan(const qst_problem_desc *probs_in, int32_t n, const qst_sampler_cfg *cfg, Plan &plan) {
    if (!probs_in || n < 1) return fail(QST_ERR_INVALID_ARG, "need at least one problem");
    qst_status st = validate_cfg(cfg);
    if (st != QST_OK) return st;
    // NULL POVM arrays select the built-in Pauli POVMs (num_povms must then be 3^Q)
    std::vector<qst_problem_desc> probs_v(probs_in, probs_in + n);
    std::vector<std::vector<double>> pauli_store;
    pauli_store.reserve(2 * (size_t)n);
    std::vector<char> builtin_in(n, 0);
    const bool autof = cfg->precision == QST_PREC_AUTO;
    for (int i = 0; i < n; ++i) {
        qst_problem_desc &d = probs_v[i];
        if (d.povm_re || d.povm_im) continue;
        builtin_in[i] = 1;
        if (d.num_qubits < 1 || d.num_qubits > max_qubits(cfg, true))
            return fail(QST_ERR_INVALID_ARG, "problem %d: num_qubits %d outside 1..%d", i, d.num_qubits,
                        max_qubits(cfg, true));
        if (d.num_povms != (int32_t)std::lround(std::pow(3.0, d.num_qubits)))
            return fail(QST_ERR_INVALID_ARG, "problem %d: the built-in Pauli POVMs need num_povms = 3^Q", i);
        if (cfg->precision == QST_PREC_PAULI) continue;   // never reads the arrays
        if (autof && d.num_qubits > 5) continue;         // only the structured form goes that far
        pauli_store.emplace_back();
        pauli_store.emplace_back();
        std::vector<double> &re = pauli_store[pauli_store.size() - 2], &im = pauli_store.back();
        pauli_povms(d.num_qubits, re, im);
        d.povm_re = re.data();
        d.povm_im = im.data();
    }
    const qst_problem_desc *probs = probs_v.data();
    plan.probs.clear();
    plan.probs.resize(n);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    for (int i = 0; i < n; ++i) {
        const qst_problem_desc &d = probs[i];
        st = validate_problem(d, i, cfg);
        if (st != QST_OK) return st;
        HostProblem &hp = plan.probs[i];
        ProblemView &v = hp.v;
        hp.Q = d.num_qubits;
        hp.K = d.num_povms;
        v.D = 1 << d.num_qubits;
        v.d = v.D * v.D;
        v.nx = 4 * v.d;
        v.KD = d.num_povms * v.D;
        v.d_pad = round_up(v.d, 64);
        v.KD_pad = round_up(v.KD, 128);
        v.R = d.num_chains;
        v.chain_offset = d.chain_offset;
        v.seed = d.seed;
        hp.beta0 = d.beta0 > 0.0 ? d.beta0 : cfg->beta0;
        int kind = tc_kind_of(cfg->precision);
        bool pauli = cfg->precision == QST_PREC_PAULI;
        if (autof) {   // the forms that apply; the choice between them comes after the packing
            hp.can_pauli = builtin_in[i] || povms_are_pauli(d);
            hp.can_tc = d.povm_re != nullptr && tc_supported(TC_BF16X3, v.D);
            kind = hp.can_tc ? TC_BF16X3 : TC_NONE;
            pauli = false;
        }
        bool tc = kind != TC_NONE;
        v.tc_kind = kind;
        v.pauli = pauli ? 1 : 0;
        if (tc) {
            const int nt = tc_column_tile(v.D, v.KD);
            if (nt <= 0) return fail(QST_ERR_UNSUPPORTED, "problem %d: no tensor-core column tile for %d projectors", i, v.KD);
            v.KD_tc = round_up(v.KD, nt);
        } else {
            v.KD_tc = 0;
        }
        hp.KDmax = std::max(v.KD_pad, v.KD_tc);
        // packed projectors
        std::vector<double> P;
        if (!pauli && d.povm_re) {   // the structured form never reads a projector matrix
            P.resize((size_t)v.d * v.KD);
            pack_projectors(v.D, v.KD, d.povm_re, d.povm_im, P.data(), v.KD);
            hp.P32.assign((size_t)v.d_pad * v.KD_pad, 0.0f);
            for (int r = 0; r < v.d; ++r)
                for (int m = 0; m < v.KD; ++m) hp.P32[(size_t)r * v.KD_pad + m] = (float)P[(size_t)r * v.KD + m];
        }
        if (kind == TC_BF16X3 && autof) {   // AUTO: the tensor-core form only where P is exact in bf16
            for (size_t e = 0; e < P.size() && hp.can_tc; ++e) hp.can_tc = bf16_exact(P[e]);
            if (!hp.can_tc) {
                kind = TC_NONE;
                tc = false;
                v.tc_kind = TC_NONE;
                v.KD_tc = 0;
                hp.KDmax = v.KD_pad;
            }
        }
        if (kind == TC_BF16X3) {
            hp.Pbf.assign((size_t)v.KD_tc * v.d_pad, __float2bfloat16_rn(0.0f));
            for (int r = 0; r < v.d; ++r)
                for (int m = 0; m < v.KD; ++m) {
                    const double x = P[(size_t)r * v.KD + m];
                    if (!bf16_exact(x))
                        return fail(QST_ERR_INVALID_ARG,
                                    "problem %d: packed projector entry %.17g is not exact in bf16; use QST_PREC_FP32",
                                    i, x);
                    hp.Pbf[(size_t)m * v.d_pad + r] = __float2bfloat16_rn((float)x);
                    hp.P32[(size_t)r * v.KD_pad + m] = __bfloat162float(hp.Pbf[(size_t)m * v.d_pad + r]);
                }
        } else if (tc) {
            hp.Ptf.assign((size_t)v.KD_tc * v.d_pad, 0.0f);
            for (int r = 0; r < v.d; ++r)
                for (int m = 0; m < v.KD; ++m) {
                    const double x = P[(size_t)r * v.KD + m];
                    if (!tf32_exact(x))
                        return fail(QST_ERR_INVALID_ARG,
                                    "problem %d: packed projector entry %.17g is not exact in TF32; use QST_PREC_FP32",
                                    i, x);
                    hp.Ptf[(size_t)m * v.d_pad + r] = (float)x;
                }
        }
        // deviance weights: log L = C0 + sum_{c>0} c log(p * invf), invf = P_k / c (as float); for
        // the Poisson likelihood invf = mu_k / c, the per-setting weight is mu_k, and C0 adds
        // sum_{c>0} c log mu_k - sum_k mu_k (the projection kernels give each setting
        // -mu_k (S_k / t - 1) in place of -P_k log(S_k / t))
        const bool poisson = d.likelihood == QST_LIKELIHOOD_POISSON;
        v.poisson = poisson ? 1 : 0;
        hp.cnt.assign(hp.KDmax, 0.0f);
        hp.invf.assign(hp.KDmax, 1.0f);
        hp.ptot.assign(hp.KDmax / v.D, 0.0f);
        double C0 = 0.0, Ntot = 0.0;
        for (int k = 0; k < d.num_povms; ++k) {
            int64_t Pk = 0;
            for (int l = 0; l < v.D; ++l) Pk += d.counts[k * v.D + l];
            const double wk = poisson ? d.trials[k] : (double)Pk;
            hp.ptot[k] = (float)wk;
            if (poisson) C0 -= wk;
            for (int l = 0; l < v.D; ++l) {
                const int m = k * v.D + l;
                const int c = d.counts[m];
                if (c == 0) continue;
                const float invf = (float)(wk / (double)c);
                hp.cnt[m] = (float)c;
                hp.invf[m] = invf;
                C0 -= (double)c * std::log((double)invf);
                if (poisson) C0 += (double)c * std::log(wk);
                Ntot += (double)c;
            }
        }
        v.C0 = C0;
        v.Ntot = Ntot;
        if (pauli || hp.can_pauli) {
            pauli_tree_order(hp.Q, hp.pauli_perm);
            pauli_weights(hp.Q, hp.pauli_perm, hp.cnt.data(), hp.invf.data(), hp.pauli_wq, hp.pauli_wc);
        }
        if (autof) {   // the rule without timing: the structured form from five qubits on or without P
            pauli = hp.can_pauli && (v.D >= 32 || !hp.can_tc);
            v.pauli = pauli ? 1 : 0;
        }
        // column groups: a fixed rule, and the candidates the autotuner may time instead
        if (tc) {
            hp.tc_groups_rule = tc_ngroups(v, v.R);
            const int ntiles = v.KD_tc / tc_column_tile(v.D, v.KD);
            if (v.D == 32) {
                hp.tc_group_choices = {hp.tc_groups_rule};
            } else {
                for (int g = 1; g < ntiles; g *= 2) hp.tc_group_choices.push_back(4 * g);
                hp.tc_group_choices.push_back(4 * ntiles);
            }
        }
        if (pauli) {
            v.ngroups = 1;
            hp.group_choices = {1};
        } else if (tc) {
            v.ngroups = hp.tc_groups_rule;
            hp.group_choices = hp.tc_group_choices;
        } else {
            v.ngroups = fp32_ngroups(v, v.R);
            const int nt = v.KD_pad / 128;
            for (int g = 1; g < nt; g *= 2) hp.group_choices.push_back(g);
            hp.group_choices.push_back(nt);
        }
        hp.part_slots = v.ngroups;
        for (int g : hp.group_choices) hp.part_slots = std::max(hp.part_slots, g);
        for (int g : hp.tc_group_choices) hp.part_slots = std::max(hp.part_slots, g);
        // the passes this problem's proposal kernel runs: 0, no QR (W = G); the refinement (3) at
        // D <= 16, and at D = 32 only when 4 is asked for; D = 64 has the first-order form (2)
        v.qr_passes = cfg->prior == QST_PRIOR_HS ? 0 : cfg->qr_passes;
        if (v.qr_passes >= 3) v.qr_passes = (v.D <= 16 || (v.D == 32 && v.qr_passes == 4)) ? 3 : 2;
        // a forced proposal CTA size (only the default QR and the Hilbert-Schmidt prior have the
        // smaller sizes; it must hold at least one chain)
        if (cfg->propose_threads != 0 && v.D <= 16 && (v.qr_passes == 0 || v.qr_passes == 3) &&
            cfg->propose_threads >= v.D)
            v.propose_threads = cfg->propose_threads;
        v.accept_cpc = accept_chains_per_cta(v.R, v.d);
        v.n_slots = (int)((v.R + v.accept_cpc - 1) / v.accept_cpc);
        v.n_diag = (int)std::min<int64_t>(cfg->diag_chains, v.R);
        v.traj_cap = cfg->traj_capacity;
        if (v.traj_cap == 0) v.n_diag = 0;
        v.trace_steps = cfg->trace_steps;
        Layout &L = hp.off;
        const int64_t R = v.R;
        L.P32 = take(sizeof(float) * hp.P32.size());
        L.Ptc = take(tc ? (size_t)tc_elem_bytes(kind) * v.KD_tc * v.d_pad : 0);
        L.cnt = take(sizeof(float) * hp.KDmax);
        L.invf = take(sizeof(float) * hp.KDmax);
        L.ptot = take(sizeof(float) * (hp.KDmax / v.D));
        L.colw = take(sizeof(float4) * (hp.KDmax / 2));
        L.pauli_wq = take(sizeof(float4) * hp.pauli_wq.size());
        L.pauli_wc = take(sizeof(float2) * hp.pauli_wc.size());
        L.pauli_perm = take(sizeof(int32_t) * hp.pauli_perm.size());
        L.y = take(sizeof(float) * 2 * R * v.nx);
        L.cur = take(R);
        L.rho_cur = take(sizeof(float) * R * v.d_pad);
        L.rho_prop = take(sizeof(float) * R * v.d_pad);
        L.rho_split = take(tc ? (size_t)tc_elem_bytes(kind) * tc_splits(kind) * R * v.d_pad : 0);
        L.trace_prop = take(sizeof(double) * R);
        L.logl_cur = take(sizeof(double) * R);
        L.logl_part = take(sizeof(double) * hp.part_slots * R);
        L.beta = take(sizeof(double) * R);
        L.coef = take(sizeof(float2) * R);
        L.acc_win = take(sizeof(int32_t) * R);
        L.acc_total = take(sizeof(int64_t) * R);
        L.pool = take(sizeof(double) * v.n_slots * v.d);
        L.traj = take(sizeof(float) * (size_t)v.n_diag * v.traj_cap * v.d);
        L.trace_acc = take((size_t)v.trace_steps * R);
        L.trace_logl = take(sizeof(double) * v.trace_steps * R);
        L.red = take(sizeof(double) * v.d);
        L.acf = take(sizeof(double) * (size_t)std::max(v.n_diag, 1) * (cfg->acf_lmax + 1));
        L.logl_eval = take(sizeof(double) * R);
        L.end = off;
    }
    plan.status_off = take(256);
    plan.step_off = take(256);
    plan.bytes = off;
    return QST_OK;
}

}  // namespace

void qst::set_last_error(const char *msg) { g_last_error = msg; }

namespace {

struct EventPair {
    cudaEvent_t a, b;
    int kind;
};

}  // namespace

struct qst_handle {
    Plan plan;
    qst_sampler_cfg cfg{};
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    uint32_t *d_status = nullptr;
    StepState *d_step = nullptr;
    cudaStream_t capture_stream = nullptr;   // private stream the step graph is captured on
    static constexpr int kBranches = 8;      // problems of a graph step run on up to 8 parallel branches
    cudaStream_t branch[kBranches] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kBranches] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_kernels = 0;               // kernel launches one replay performs
    int64_t steps_done = 0;
    int64_t kept = 0;
    int64_t launches = 0;
    bool prof = false;
    std::vector<EventPair> pending;
    std::vector<EventPair> spare;
    double kind_ms[QST_KERNEL_KINDS] = {0, 0, 0, 0};
    int64_t kind_launches[QST_KERNEL_KINDS] = {0, 0, 0, 0};
    SamplerParams sp{};
};

namespace {

template <class F>
qst_status launch(qst_handle *h, int kind, const char *what, F &&f) {
    EventPair ev{};
    if (h->prof) {
        if (!h->spare.empty()) {
            ev = h->spare.back();
            h->spare.pop_back();
        } else {
            QST_CUDA(cudaEventCreate(&ev.a), "cudaEventCreate");
            QST_CUDA(cudaEventCreate(&ev.b), "cudaEventCreate");
        }
        ev.kind = kind;
        QST_CUDA(cudaEventRecord(ev.a, h->stream), "cudaEventRecord");
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (h->prof) {
        QST_CUDA(cudaEventRecord(ev.b, h->stream), "cudaEventRecord");
        h->pending.push_back(ev);
    }
    h->launches += 1;
    h->kind_launches[kind] += 1;
    return QST_OK;
}

qst_status harvest(qst_handle *h) {
    for (auto &ev : h->pending) {
        QST_CUDA(cudaEventSynchronize(ev.b), "cudaEventSynchronize");
        float ms = 0.0f;
        QST_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b), "cudaEventElapsedTime");
        h->kind_ms[ev.kind] += ms;
        h->spare.push_back(ev);
    }
    h->pending.clear();
    return QST_OK;
}

qst_status check_status(qst_handle *h) {
    QST_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    uint32_t st = 0;
    QST_CUDA(cudaMemcpy(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost), "read status");
    if (st & STATUS_TIMEOUT) return fail(QST_ERR_TIMEOUT, "a device wait gave up (status 0x%x)", st);
    if (st & (STATUS_BOUNDS | STATUS_BAD_LAUNCH)) return fail(QST_ERR_NUMERIC, "device check failed (status 0x%x)", st);
    return QST_OK;
}

qst_status bind_problem(qst_handle *h, HostProblem &hp) {
    char *b = h->ws;
    ProblemView &v = hp.v;
    const Layout &L = hp.off;
    v.P32 = reinterpret_cast<const float *>(b + L.P32);
    v.Ptc = b + L.Ptc;
    v.cnt = reinterpret_cast<const float *>(b + L.cnt);
    v.invf = reinterpret_cast<const float *>(b + L.invf);
    v.ptot = reinterpret_cast<const float *>(b + L.ptot);
    v.colw = reinterpret_cast<const float4 *>(b + L.colw);
    const bool pauli_buffers = !hp.pauli_wq.empty();
    v.pauli_wq = pauli_buffers ? reinterpret_cast<const float4 *>(b + L.pauli_wq) : nullptr;
    v.pauli_wc = pauli_buffers ? reinterpret_cast<const float2 *>(b + L.pauli_wc) : nullptr;
    v.pauli_perm = pauli_buffers ? reinterpret_cast<const int32_t *>(b + L.pauli_perm) : nullptr;
    v.y = reinterpret_cast<float *>(b + L.y);
    v.cur = reinterpret_cast<uint8_t *>(b + L.cur);
    v.rho_cur = reinterpret_cast<float *>(b + L.rho_cur);
    v.rho_prop = reinterpret_cast<float *>(b + L.rho_prop);
    v.rho_split = b + L.rho_split;
    v.trace_prop = reinterpret_cast<double *>(b + L.trace_prop);
    v.logl_cur = reinterpret_cast<double *>(b + L.logl_cur);
    v.logl_part = reinterpret_cast<double *>(b + L.logl_part);
    v.beta = reinterpret_cast<double *>(b + L.beta);
    v.coef = reinterpret_cast<float2 *>(b + L.coef);
    v.acc_win = reinterpret_cast<int32_t *>(b + L.acc_win);
    v.acc_total = reinterpret_cast<int64_t *>(b + L.acc_total);
    v.pool = reinterpret_cast<double *>(b + L.pool);
    v.traj = reinterpret_cast<float *>(b + L.traj);
    v.trace_acc = reinterpret_cast<uint8_t *>(b + L.trace_acc);
    v.trace_logl = reinterpret_cast<double *>(b + L.trace_logl);
    return QST_OK;
}

// the problem's projection runs on the tensor cores (and so needs the split operand)
bool uses_tc(const ProblemView &v) { return v.tc_kind != TC_NONE && !v.pauli; }

// proposal -> projection -> (accept) for one problem
qst_status enqueue_projection(qst_handle *h, HostProblem &hp, int64_t rows, float *p_out) {
    ProblemView &v = hp.v;
    if (v.pauli) {
        return launch(h, QST_KERNEL_PROJECT, "projection (structured Pauli)", [&] {
            return launch_project_pauli(v, v.rho_prop, rows, v.logl_part, p_out, h->stream);
        });
    }
    if (v.tc_kind != TC_NONE) {
        return launch(h, QST_KERNEL_PROJECT, "projection (tcgen05)", [&] {
            return launch_project_tc(hp.tc, v, rows, v.logl_part, p_out, h->d_status, h->stream);
        });
    }
    return launch(h, QST_KERNEL_PROJECT, "projection (fp32)", [&] {
        return launch_project_fp32(v, v.rho_prop, rows, v.logl_part, p_out, h->stream);
    });
}

qst_status enqueue_init(qst_handle *h, HostProblem &hp) {
    ProblemView &v = hp.v;
    qst_status st = launch(h, QST_KERNEL_PROPOSE, "propose (init)", [&] {
        return launch_propose(v, MODE_INIT, 0u, nullptr, nullptr, 0, uses_tc(v), nullptr, h->d_status, h->stream);
    });
    if (st != QST_OK) return st;
    st = enqueue_projection(h, hp, v.R, nullptr);
    if (st != QST_OK) return st;
    return launch(h, QST_KERNEL_ACCEPT, "accept (init)", [&] {
        return launch_accept(v, h->sp, MODE_INIT, nullptr, 0u, false, 0, h->d_status, h->stream);
    });
}

}  // namespace

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

const char *qst_status_string(qst_status s) {
    switch (s) {
        case QST_OK: return "ok";
        case QST_ERR_INVALID_ARG: return "invalid argument";
        case QST_ERR_CUDA: return "CUDA error";
        case QST_ERR_OOM: return "out of memory";
        case QST_ERR_TIMEOUT: return "device wait timed out";
        case QST_ERR_NUMERIC: return "numeric or device check failure";
        case QST_ERR_STATE: return "invalid state";
        case QST_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *qst_last_error(void) { return g_last_error.c_str(); }

void qst_default_config(qst_sampler_cfg *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->beta0 = 0.1;
    cfg->adapt_interval = 500;
    cfg->acc_lo = 0.2;
    cfg->acc_hi = 0.6;
    cfg->adapt_factor = 1.1;
    cfg->beta_max = 1.0;
    cfg->thin = 1;
    cfg->burn_in = 0;
    cfg->diag_chains = 256;
    cfg->traj_capacity = 1024;
    cfg->acf_lmax = 200;
    cfg->trace_steps = 0;
    cfg->precision = QST_PREC_FP32;
    cfg->qr_passes = 3;
    cfg->use_graph = 1;
    cfg->autotune = 1;
    cfg->propose_threads = 0;
}

qst_status qst_workspace_size(const qst_problem_desc *problems, int32_t num_problems, const qst_sampler_cfg *cfg,
                              size_t *bytes) {
    if (!bytes) return fail(QST_ERR_INVALID_ARG, "bytes is NULL");
    Plan plan;
    qst_status st = make_plan(problems, num_problems, cfg, plan);
    if (st != QST_OK) return st;
    *bytes = plan.bytes;
    return QST_OK;
}

namespace {

// QST_PREC_AUTO: for every problem whose projection can run both on the tensor cores and in
// the structured Pauli form, times both (each on its rule's column groups, one warm-up launch
// and three timed ones, on a fresh step-1 proposal that carries the tensor cores' split
// operand) and keeps the faster.  A problem whose form changes is initialised again, so that
// the cached log L of its current state comes from the form it will run.
qst_status autotune_form(qst_handle *h) {
    if (h->cfg.precision != QST_PREC_AUTO) return QST_OK;
    cudaEvent_t e0, e1;
    QST_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    QST_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    qst_status st = QST_OK;
    for (auto &hp : h->plan.probs) {
        ProblemView &v = hp.v;
        if (!(hp.can_tc && hp.can_pauli)) continue;
        const int first = v.pauli;
        v.pauli = 0;
        st = launch(h, QST_KERNEL_PROPOSE, "autotune form (proposal)", [&] {
            return launch_propose(v, MODE_STEP, 1u, nullptr, nullptr, 0, true, nullptr, h->d_status, h->stream);
        });
        float ms[2] = {0.0f, 0.0f};
        for (int f = 0; f < 2 && st == QST_OK; ++f) {
            v.pauli = f;   // 0: tensor cores, 1: structured Pauli
            v.ngroups = f ? 1 : hp.tc_groups_rule;
            st = enqueue_projection(h, hp, v.R, nullptr);
            if (st != QST_OK) break;
            if (cudaEventRecord(e0, h->stream) != cudaSuccess) { st = fail(QST_ERR_CUDA, "autotune: event"); break; }
            for (int r = 0; r < 3 && st == QST_OK; ++r) st = enqueue_projection(h, hp, v.R, nullptr);
            if (st != QST_OK) break;
            if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms[f], e0, e1) != cudaSuccess)
                st = fail(QST_ERR_CUDA, "autotune: timing");
        }
        if (st != QST_OK) break;
        v.pauli = ms[1] < ms[0] ? 1 : 0;
        v.ngroups = v.pauli ? 1 : hp.tc_groups_rule;
        hp.group_choices = v.pauli ? std::vector<int>{1} : hp.tc_group_choices;
        if (v.pauli != first) {
            st = enqueue_init(h, hp);
            if (st != QST_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Times the projection of every problem with each candidate column-group count (one warm-up
// launch, then three timed ones on the handle's stream, on the proposal buffers that hold
// rho(y0) after initialisation) and keeps the fastest.  Only the schedule changes: every
// candidate computes the same partial sums, split differently over CTAs.
qst_status autotune_groups(qst_handle *h) {
    cudaEvent_t e0, e1;
    QST_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    QST_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    qst_status st = QST_OK;
    for (auto &hp : h->plan.probs) {
        if (hp.group_choices.size() < 2) continue;
        int best = hp.v.ngroups;
        float best_ms = 0.0f;
        for (int g : hp.group_choices) {
            hp.v.ngroups = g;
            st = enqueue_projection(h, hp, hp.v.R, nullptr);
            if (st != QST_OK) break;
            if (cudaEventRecord(e0, h->stream) != cudaSuccess) { st = fail(QST_ERR_CUDA, "autotune: event"); break; }
            for (int r = 0; r < 3 && st == QST_OK; ++r) st = enqueue_projection(h, hp, hp.v.R, nullptr);
            if (st != QST_OK) break;
            float ms = 0.0f;
            if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = fail(QST_ERR_CUDA, "autotune: timing");
                break;
            }
            if (best_ms == 0.0f || ms < best_ms) {
                best_ms = ms;
                best = g;
            }
        }
        hp.v.ngroups = best;
        if (st != QST_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Times the proposal kernel of every problem of 1-4 qubits with 128-, 64- and 32-thread CTAs
// (16, 8, 4 ... chains per CTA at four qubits) and keeps the fastest.  A problem whose
// 128-thread grid already fills every SM twice keeps 128 untimed.  The proposal writes only
// the proposal buffers, which hold nothing the chains need between steps, so the timing
// launches (step 1, one warm-up and three timed) change no chain state.
qst_status autotune_propose(qst_handle *h) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0)
        sms = 148;
    cudaEvent_t e0, e1;
    QST_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    QST_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    qst_status st = QST_OK;
    for (auto &hp : h->plan.probs) {
        ProblemView &v = hp.v;
        if (v.D > 16 || (v.qr_passes != 0 && v.qr_passes != 3) || h->cfg.propose_threads != 0) continue;
        const int64_t blocks128 = (v.R + 128 / v.D - 1) / (128 / v.D);
        if (blocks128 >= 2 * 5 * (int64_t)sms) continue;
        int best = 128;
        float best_ms = 0.0f;
        for (int threads : {128, 64, 32}) {
            if (threads < v.D) continue;
            v.propose_threads = threads;
            auto run = [&] {
                return launch(h, QST_KERNEL_PROPOSE, "autotune propose", [&] {
                    return launch_propose(v, MODE_STEP, 1u, nullptr, nullptr, 0, uses_tc(v), nullptr, h->d_status,
                                          h->stream);
                });
            };
            st = run();
            if (st != QST_OK) break;
            if (cudaEventRecord(e0, h->stream) != cudaSuccess) { st = fail(QST_ERR_CUDA, "autotune: event"); break; }
            for (int r = 0; r < 3 && st == QST_OK; ++r) st = run();
            if (st != QST_OK) break;
            float ms = 0.0f;
            if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = fail(QST_ERR_CUDA, "autotune: timing");
                break;
            }
            if (best_ms == 0.0f || ms < best_ms) {
                best_ms = ms;
                best = threads;
            }
        }
        v.propose_threads = best;
        if (st != QST_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace

qst_status qst_create(const qst_problem_desc *problems, int32_t num_problems, const qst_sampler_cfg *cfg,
                      void *d_workspace, size_t workspace_bytes, void *cuda_stream, qst_handle **out) {
    if (!out) return fail(QST_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::unique_ptr<qst_handle> h(new qst_handle());
    qst_status st = make_plan(problems, num_problems, cfg, h->plan);
    if (st != QST_OK) return st;
    h->cfg = *cfg;
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    h->sp.adapt_interval = cfg->adapt_interval;
    h->sp.acc_lo = cfg->acc_lo;
    h->sp.acc_hi = cfg->acc_hi;
    h->sp.adapt_factor = cfg->adapt_factor;
    h->sp.beta_max = cfg->beta_max;
    if (d_workspace) {
        if (workspace_bytes < h->plan.bytes)
            return fail(QST_ERR_OOM, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
                        h->plan.bytes);
        if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
            return fail(QST_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        h->ws = static_cast<char *>(d_workspace);
        h->ws_bytes = workspace_bytes;
    } else {
        void *p = nullptr;
        QST_CUDA(cudaMalloc(&p, h->plan.bytes), "cudaMalloc(workspace)");
        h->ws = static_cast<char *>(p);
        h->ws_bytes = h->plan.bytes;
        h->own_ws = true;
    }
    QST_CUDA(cudaMemsetAsync(h->ws, 0, h->plan.bytes, h->stream), "clear workspace");
    h->d_status = reinterpret_cast<uint32_t *>(h->ws + h->plan.status_off);
    h->d_step = reinterpret_cast<StepState *>(h->ws + h->plan.step_off);
    for (auto &hp : h->plan.probs) {
        bind_problem(h.get(), hp);
        ProblemView &v = hp.v;
        const Layout &L = hp.off;
        QST_CUDA(cudaMemcpyAsync(h->ws + L.P32, hp.P32.data(), sizeof(float) * hp.P32.size(), cudaMemcpyHostToDevice,
                                 h->stream), "upload P");
        if (!hp.pauli_wq.empty()) {
            QST_CUDA(cudaMemcpyAsync(h->ws + L.pauli_wq, hp.pauli_wq.data(), sizeof(float4) * hp.pauli_wq.size(),
                                     cudaMemcpyHostToDevice, h->stream), "upload deviance weights");
            QST_CUDA(cudaMemcpyAsync(h->ws + L.pauli_wc, hp.pauli_wc.data(), sizeof(float2) * hp.pauli_wc.size(),
                                     cudaMemcpyHostToDevice, h->stream), "upload counts (pairs)");
            QST_CUDA(cudaMemcpyAsync(h->ws + L.pauli_perm, hp.pauli_perm.data(),
                                     sizeof(int32_t) * hp.pauli_perm.size(), cudaMemcpyHostToDevice, h->stream),
                     "upload tree order");
        }
        if (!hp.Pbf.empty())
            QST_CUDA(cudaMemcpyAsync(h->ws + L.Ptc, hp.Pbf.data(), sizeof(__nv_bfloat16) * hp.Pbf.size(),
                                     cudaMemcpyHostToDevice, h->stream), "upload P (bf16)");
        if (!hp.Ptf.empty())
            QST_CUDA(cudaMemcpyAsync(h->ws + L.Ptc, hp.Ptf.data(), sizeof(float) * hp.Ptf.size(),
                                     cudaMemcpyHostToDevice, h->stream), "upload P (TF32)");
        QST_CUDA(cudaMemcpyAsync(h->ws + L.cnt, hp.cnt.data(), sizeof(float) * hp.KDmax, cudaMemcpyHostToDevice,
                                 h->stream), "upload counts");
        QST_CUDA(cudaMemcpyAsync(h->ws + L.invf, hp.invf.data(), sizeof(float) * hp.KDmax, cudaMemcpyHostToDevice,
                                 h->stream), "upload weights");
        QST_CUDA(cudaMemcpyAsync(h->ws + L.ptot, hp.ptot.data(), sizeof(float) * hp.ptot.size(), cudaMemcpyHostToDevice,
                                 h->stream), "upload setting totals");
        // per column pair (2p, 2p+1): (invf, invf, add, add) with x = q invf + add; a column
        // without counts gets invf = 0, add = 1, so its log is exactly 0
        std::vector<float4> colw(hp.KDmax / 2);
        for (int m = 0; m < hp.KDmax; m += 2) {
            const bool c0 = hp.cnt[m] > 0.0f, c1 = hp.cnt[m + 1] > 0.0f;
            colw[m / 2] = make_float4(c0 ? hp.invf[m] : 0.0f, c1 ? hp.invf[m + 1] : 0.0f, c0 ? 0.0f : 1.0f,
                                      c1 ? 0.0f : 1.0f);
        }
        QST_CUDA(cudaMemcpyAsync(h->ws + L.colw, colw.data(), sizeof(float4) * colw.size(), cudaMemcpyHostToDevice,
                                 h->stream), "upload column weights");
        std::vector<double> beta(v.R, hp.beta0);
        QST_CUDA(cudaMemcpyAsync(v.beta, beta.data(), sizeof(double) * v.R, cudaMemcpyHostToDevice, h->stream),
                 "upload beta");
        std::vector<float2> coef(v.R, make_float2((float)std::sqrt(1.0 - hp.beta0 * hp.beta0), (float)hp.beta0));
        QST_CUDA(cudaMemcpyAsync(v.coef, coef.data(), sizeof(float2) * v.R, cudaMemcpyHostToDevice, h->stream),
                 "upload proposal coefficients");
        // pageable copies above are staged synchronously; keep the host vectors alive until then
        QST_CUDA(cudaStreamSynchronize(h->stream), "stream sync");
        if (v.tc_kind != TC_NONE) {
            cudaError_t e = tc_plan_create(v, v.rho_split, v.R, &hp.tc);
            if (e != cudaSuccess) return cuda_fail(e, "tensor-core plan");
        }
        st = enqueue_init(h.get(), hp);
        if (st != QST_OK) return st;
        std::vector<float>().swap(hp.P32);
        std::vector<__nv_bfloat16>().swap(hp.Pbf);
        std::vector<float>().swap(hp.Ptf);
    }
    if (cfg->autotune) {
        st = autotune_form(h.get());
        if (st == QST_OK) st = autotune_groups(h.get());
        if (st == QST_OK) st = autotune_propose(h.get());
        if (st != QST_OK) return st;
    }
    *out = h.release();
    return QST_OK;
}

namespace {

// One step's launches on h->stream: open step j on the device, then every problem's
// proposal, projection and accept, all reading j from the device.  With `branches` (graph
// capture) the problems are spread over parallel branches -- they are independent -- so
// the graph runs the kernels of different problems concurrently.
qst_status enqueue_problem(qst_handle *h, HostProblem &hp) {
    ProblemView &v = hp.v;
    qst_status st = launch(h, QST_KERNEL_PROPOSE, "propose", [&] {
        return launch_propose(v, MODE_STEP, 0u, h->d_step, nullptr, 0, uses_tc(v), nullptr, h->d_status, h->stream);
    });
    if (st != QST_OK) return st;
    st = enqueue_projection(h, hp, v.R, nullptr);
    if (st != QST_OK) return st;
    return launch(h, QST_KERNEL_ACCEPT, "accept", [&] {
        return launch_accept(v, h->sp, MODE_STEP, h->d_step, 0u, false, 0, h->d_status, h->stream);
    });
}

qst_status enqueue_step(qst_handle *h, bool branches) {
    qst_status st = launch(h, QST_KERNEL_ACCEPT, "advance step",
                           [&] { return launch_advance_step(h->d_step, h->cfg.thin, h->cfg.burn_in, h->stream); });
    if (st != QST_OK) return st;
    const int np = (int)h->plan.probs.size();
    if (!branches || np == 1) {
        for (auto &hp : h->plan.probs) {
            st = enqueue_problem(h, hp);
            if (st != QST_OK) return st;
        }
        return QST_OK;
    }
    const int nb = np < qst_handle::kBranches ? np : qst_handle::kBranches;
    cudaStream_t origin = h->stream;
    QST_CUDA(cudaEventRecord(h->fork_ev, origin), "fork");
    for (int b = 0; b < nb; ++b) QST_CUDA(cudaStreamWaitEvent(h->branch[b], h->fork_ev, 0), "branch wait");
    for (int i = 0; i < np && st == QST_OK; ++i) {
        h->stream = h->branch[i % nb];
        st = enqueue_problem(h, h->plan.probs[i]);
    }
    h->stream = origin;
    if (st != QST_OK) return st;
    for (int b = 0; b < nb; ++b) {
        QST_CUDA(cudaEventRecord(h->join_ev[b], h->branch[b]), "join");
        QST_CUDA(cudaStreamWaitEvent(origin, h->join_ev[b], 0), "join wait");
    }
    return QST_OK;
}

// Captures enqueue_step once on the private capture stream and instantiates it.
qst_status build_step_graph(qst_handle *h) {
    if (!h->capture_stream) {
        QST_CUDA(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking), "create capture stream");
        for (int b = 0; b < qst_handle::kBranches; ++b) {
            QST_CUDA(cudaStreamCreateWithFlags(&h->branch[b], cudaStreamNonBlocking), "create branch stream");
            QST_CUDA(cudaEventCreateWithFlags(&h->join_ev[b], cudaEventDisableTiming), "create event");
        }
        QST_CUDA(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming), "create event");
    }
    cudaStream_t user = h->stream;
    const int64_t launches0 = h->launches;
    h->stream = h->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
    qst_status st = QST_OK;
    if (e == cudaSuccess) st = enqueue_step(h, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = (e == cudaSuccess) ? cudaStreamEndCapture(h->capture_stream, &g) : e;
    h->stream = user;
    h->graph_kernels = h->launches - launches0;
    h->launches = launches0;
    if (e != cudaSuccess) return cuda_fail(e, "begin graph capture");
    if (st != QST_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e_end != cudaSuccess) return cuda_fail(e_end, "end graph capture");
    h->graph = g;
    QST_CUDA(cudaGraphInstantiate(&h->graph_exec, g, 0), "instantiate step graph");
    return QST_OK;
}

}  // namespace

qst_status qst_run_chains(qst_handle *h, int64_t num_steps) {
    if (!h) return fail(QST_ERR_INVALID_ARG, "handle is NULL");
    if (num_steps < 0) return fail(QST_ERR_INVALID_ARG, "num_steps must be >= 0");
    if (h->steps_done + num_steps > 0xffffffffLL) return fail(QST_ERR_INVALID_ARG, "step counter exceeds 32 bits");
    const bool graph = h->cfg.use_graph && !h->prof && num_steps > 0;
    if (graph && !h->graph_exec) {
        qst_status st = build_step_graph(h);
        if (st != QST_OK) return st;
    }
    for (int64_t s = 0; s < num_steps; ++s) {
        const int64_t j = h->steps_done + 1;
        const bool kept = (j % h->cfg.thin == 0) && (j > h->cfg.burn_in);   // mirrors advance_step_kernel
        if (graph) {
            QST_CUDA(cudaGraphLaunch(h->graph_exec, h->stream), "launch step graph");
            h->launches += h->graph_kernels;
        } else {
            qst_status st = enqueue_step(h, false);
            if (st != QST_OK) return st;
        }
        h->steps_done = j;
        if (kept) h->kept += 1;
    }
    return QST_OK;
}

static qst_status get_problem(qst_handle *h, int32_t problem, HostProblem **hp) {
    if (!h) return fail(QST_ERR_INVALID_ARG, "handle is NULL");
    if (problem < 0 || problem >= (int32_t)h->plan.probs.size())
        return fail(QST_ERR_INVALID_ARG, "problem index %d out of range", problem);
    *hp = &h->plan.probs[problem];
    return QST_OK;
}

// The FP64 sum of the kept packed states of one problem (d doubles, host) and their count.
static qst_status pooled_sum(qst_handle *h, int32_t problem, std::vector<double> &sum, int64_t &n, int &D) {
    HostProblem *hp;
    qst_status st = get_problem(h, problem, &hp);
    if (st != QST_OK) return st;
    const ProblemView &v = hp->v;
    n = h->kept * v.R;
    D = v.D;
    if (n == 0) return fail(QST_ERR_STATE, "no state has been pooled yet");
    double *red = reinterpret_cast<double *>(h->ws + hp->off.red);
    st = launch(h, QST_KERNEL_DIAG, "pool reduce", [&] { return launch_pool_reduce(v, red, h->stream); });
    if (st != QST_OK) return st;
    sum.assign(v.d, 0.0);
    QST_CUDA(cudaMemcpyAsync(sum.data(), red, sizeof(double) * v.d, cudaMemcpyDeviceToHost, h->stream), "read pool");
    return check_status(h);
}

qst_status qst_posterior_sum(qst_handle *h, int32_t problem, double *sum_packed, int64_t *num_pooled) {
    std::vector<double> sum;
    int64_t n = 0;
    int D = 0;
    if (num_pooled) *num_pooled = 0;
    qst_status st = pooled_sum(h, problem, sum, n, D);
    if (num_pooled) *num_pooled = n;
    if (st != QST_OK) return st;
    if (sum_packed) std::memcpy(sum_packed, sum.data(), sizeof(double) * sum.size());
    return QST_OK;
}

qst_status qst_posterior_mean(qst_handle *h, int32_t problem, double *rho_re, double *rho_im, int64_t *num_pooled) {
    std::vector<double> sum;
    int64_t n = 0;
    int D = 0;
    if (num_pooled) *num_pooled = 0;
    qst_status st = pooled_sum(h, problem, sum, n, D);
    if (num_pooled) *num_pooled = n;
    if (st != QST_OK) return st;
    for (int i = 0; i < D; ++i)
        for (int j = i; j < D; ++j) {
            const double re = sum[i * D + j] / (double)n;
            const double im = (i < j) ? -sum[j * D + i] / (double)n : 0.0;
            if (rho_re) {
                rho_re[i * D + j] = re;
                rho_re[j * D + i] = re;
            }
            if (rho_im) {
                rho_im[i * D + j] = im;
                rho_im[j * D + i] = -im;
            }
        }
    return QST_OK;
}

qst_status qst_diagnostics(qst_handle *h, int32_t problem, qst_diag *out, double *acf, double *tau) {
    HostProblem *hp;
    qst_status st = get_problem(h, problem, &hp);
    if (st != QST_OK) return st;
    if (!out) return fail(QST_ERR_INVALID_ARG, "out is NULL");
    const ProblemView &v = hp->v;
    std::memset(out, 0, sizeof(*out));
    out->steps_done = h->steps_done;
    out->num_kept = h->kept;
    out->num_pooled = h->kept * v.R;
    out->acf_lmax = h->cfg.acf_lmax;
    std::vector<double> beta(v.R), logl(v.R);
    std::vector<int64_t> acc(v.R);
    QST_CUDA(cudaMemcpyAsync(beta.data(), v.beta, sizeof(double) * v.R, cudaMemcpyDeviceToHost, h->stream), "read beta");
    QST_CUDA(cudaMemcpyAsync(logl.data(), v.logl_cur, sizeof(double) * v.R, cudaMemcpyDeviceToHost, h->stream), "read logl");
    QST_CUDA(cudaMemcpyAsync(acc.data(), v.acc_total, sizeof(int64_t) * v.R, cudaMemcpyDeviceToHost, h->stream), "read acc");
    const int lmax = h->cfg.acf_lmax;
    const int n_kept = (int)std::min<int64_t>(h->kept, v.traj_cap);
    const bool do_acf = v.n_diag > 0 && n_kept > lmax;
    std::vector<double> raw;
    if (do_acf) {
        double *acf_dev = reinterpret_cast<double *>(h->ws + hp->off.acf);
        st = launch(h, QST_KERNEL_DIAG, "acf", [&] { return launch_acf(v, n_kept, lmax, acf_dev, h->stream); });
        if (st != QST_OK) return st;
        raw.resize((size_t)v.n_diag * (lmax + 1));
        QST_CUDA(cudaMemcpyAsync(raw.data(), acf_dev, sizeof(double) * raw.size(), cudaMemcpyDeviceToHost, h->stream),
                 "read acf");
    }
    st = check_status(h);
    uint32_t status = 0;
    cudaMemcpy(&status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost);
    out->device_status = status;
    out->column_groups = (uint32_t)(uses_tc(hp->v) ? hp->v.ngroups / 4 : hp->v.ngroups);
    out->projection_form = v.pauli ? QST_PREC_PAULI : uses_tc(v) ? h->cfg.precision == QST_PREC_AUTO
                                                                        ? (int32_t)QST_PREC_BF16X3
                                                                        : h->cfg.precision
                                                 : (int32_t)QST_PREC_FP32;
    out->propose_chains_per_cta =
        (uint32_t)(v.D <= 16 ? v.propose_threads / v.D : (v.D == 32 ? (v.qr_passes == 3 ? 2 : 4) : 1));
    out->qr_passes = v.qr_passes;
    out->accept_chains_per_cta = (uint32_t)v.accept_cpc;
    if (st != QST_OK) return st;
    double bmin = 1e300, bmax = -1e300, bsum = 0.0;
    int64_t acc_sum = 0, nonfinite = 0;
    for (int64_t r = 0; r < v.R; ++r) {
        bmin = std::min(bmin, beta[r]);
        bmax = std::max(bmax, beta[r]);
        bsum += beta[r];
        acc_sum += acc[r];
        if (!std::isfinite(logl[r])) nonfinite += 1;
    }
    out->beta_min = bmin;
    out->beta_max = bmax;
    out->beta_mean = bsum / (double)v.R;
    out->accept_rate = h->steps_done > 0 ? (double)acc_sum / ((double)h->steps_done * (double)v.R) : 0.0;
    out->num_nonfinite = nonfinite;
    if (do_acf) {
        out->diag_chains = v.n_diag;
        std::vector<double> mean_c(lmax + 1, 0.0);
        double tsum = 0.0, tmax = -1e300;
        int used = 0;
        for (int c = 0; c < v.n_diag; ++c) {
            const double *rc = &raw[(size_t)c * (lmax + 1)];
            if (!(rc[0] > 0.0)) {
                if (tau) tau[c] = NAN;
                continue;
            }
            double t = 1.0;
            for (int l = 1; l <= lmax; ++l) t += 2.0 * rc[l] / rc[0];
            for (int l = 0; l <= lmax; ++l) mean_c[l] += rc[l] / rc[0];
            if (tau) tau[c] = t;
            tsum += t;
            tmax = std::max(tmax, t);
            used += 1;
        }
        if (used > 0) {
            out->tau_mean = tsum / used;
            out->tau_max = tmax;
            out->n_eff = (double)out->num_pooled / out->tau_mean;
            if (acf)
                for (int l = 0; l <= lmax; ++l) acf[l] = mean_c[l] / used;
        }
        out->diag_chains = used;
    }
    return QST_OK;
}

qst_status qst_synchronize(qst_handle *h) {
    if (!h) return fail(QST_ERR_INVALID_ARG, "handle is NULL");
    return check_status(h);
}

void qst_destroy(qst_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto &hp : h->plan.probs)
        if (hp.tc) tc_plan_destroy(hp.tc);
    for (auto &ev : h->pending) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    for (auto &ev : h->spare) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (int b = 0; b < qst_handle::kBranches; ++b) {
        if (h->branch[b]) cudaStreamDestroy(h->branch[b]);
        if (h->join_ev[b]) cudaEventDestroy(h->join_ev[b]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->own_ws) cudaFree(h->ws);
    delete h;
}

qst_status qst_get_state(qst_handle *h, int32_t problem, float *y, double *logl, double *beta, int64_t *accepts) {
    HostProblem *hp;
    qst_status st = get_problem(h, problem, &hp);
    if (st != QST_OK) return st;
    const ProblemView &v = hp->v;
    if (y) {
        std::vector<uint8_t> cur(v.R);
        QST_CUDA(cudaMemcpyAsync(cur.data(), v.cur, v.R, cudaMemcpyDeviceToHost, h->stream), "read cur");
        QST_CUDA(cudaStreamSynchronize(h->stream), "sync");
        for (int64_t r = 0; r < v.R; ++r)
            QST_CUDA(cudaMemcpyAsync(y + r * v.nx, v.y + ((int64_t)cur[r] * v.R + r) * v.nx, sizeof(float) * v.nx,
                                     cudaMemcpyDeviceToHost, h->stream), "read y");
    }
    if (logl) QST_CUDA(cudaMemcpyAsync(logl, v.logl_cur, sizeof(double) * v.R, cudaMemcpyDeviceToHost, h->stream), "read logl");
    if (beta) QST_CUDA(cudaMemcpyAsync(beta, v.beta, sizeof(double) * v.R, cudaMemcpyDeviceToHost, h->stream), "read beta");
    if (accepts)
        QST_CUDA(cudaMemcpyAsync(accepts, v.acc_total, sizeof(int64_t) * v.R, cudaMemcpyDeviceToHost, h->stream),
                 "read accepts");
    return check_status(h);
}

qst_status qst_get_trace(qst_handle *h, int32_t problem, uint8_t *accept, double *logl_prop) {
    HostProblem *hp;
    qst_status st = get_problem(h, problem, &hp);
    if (st != QST_OK) return st;
    const ProblemView &v = hp->v;
    const size_t n = (size_t)v.trace_steps * v.R;
    if (accept && n) QST_CUDA(cudaMemcpyAsync(accept, v.trace_acc, n, cudaMemcpyDeviceToHost, h->stream), "read trace");
    if (logl_prop && n)
        QST_CUDA(cudaMemcpyAsync(logl_prop, v.trace_logl, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream),
                 "read trace");
    return check_status(h);
}

// Checkpoint: header (steps, kept) then every problem's state region [y .. end).
static size_t state_bytes(const HostProblem &hp) { return hp.off.end - hp.off.y; }

qst_status qst_checkpoint_size(qst_handle *h, size_t *bytes) {
    if (!h || !bytes) return fail(QST_ERR_INVALID_ARG, "NULL argument");
    size_t n = 2 * sizeof(int64_t);
    for (auto &hp : h->plan.probs) n += state_bytes(hp);
    *bytes = n;
    return QST_OK;
}

qst_status qst_checkpoint(qst_handle *h, void *buffer, size_t bytes) {
    size_t need = 0;
    qst_status st = qst_checkpoint_size(h, &need);
    if (st != QST_OK) return st;
    if (!buffer || bytes < need) return fail(QST_ERR_INVALID_ARG, "checkpoint buffer needs %zu bytes", need);
    char *p = static_cast<char *>(buffer);
    std::memcpy(p, &h->steps_done, sizeof(int64_t));
    std::memcpy(p + sizeof(int64_t), &h->kept, sizeof(int64_t));
    p += 2 * sizeof(int64_t);
    for (auto &hp : h->plan.probs) {
        QST_CUDA(cudaMemcpyAsync(p, h->ws + hp.off.y, state_bytes(hp), cudaMemcpyDeviceToHost, h->stream),
                 "checkpoint copy");
        p += state_bytes(hp);
    }
    return check_status(h);
}

qst_status qst_restore(qst_handle *h, const void *buffer, size_t bytes) {
    size_t need = 0;
    qst_status st = qst_checkpoint_size(h, &need);
    if (st != QST_OK) return st;
    if (!buffer || bytes != need) return fail(QST_ERR_INVALID_ARG, "checkpoint must be exactly %zu bytes", need);
    const char *p = static_cast<const char *>(buffer);
    int64_t steps, kept;
    std::memcpy(&steps, p, sizeof(int64_t));
    std::memcpy(&kept, p + sizeof(int64_t), sizeof(int64_t));
    p += 2 * sizeof(int64_t);
    QST_CUDA(cudaStreamSynchronize(h->stream), "sync");
    for (auto &hp : h->plan.probs) {
        QST_CUDA(cudaMemcpy(h->ws + hp.off.y, p, state_bytes(hp), cudaMemcpyHostToDevice), "restore copy");
        p += state_bytes(hp);
    }
    h->steps_done = steps;
    h->kept = kept;
    StepState ss{};
    ss.step = (uint32_t)steps;
    ss.kept_count = kept;
    QST_CUDA(cudaMemcpy(h->d_step, &ss, sizeof(ss), cudaMemcpyHostToDevice), "restore step counter");
    return check_status(h);
}

qst_status qst_evaluate(qst_handle *h, int32_t problem, const float *x, int64_t n, float *rho, float *p, double *logl) {
    HostProblem *hp;
    qst_status st = get_problem(h, problem, &hp);
    if (st != QST_OK) return st;
    ProblemView &v = hp->v;
    if (n < 0 || n > v.R) return fail(QST_ERR_INVALID_ARG, "n must be in [0, num_chains]");
    if (n == 0) return QST_OK;
    if (!x) return fail(QST_ERR_INVALID_ARG, "x is NULL");
    st = launch(h, QST_KERNEL_PROPOSE, "propose (eval)", [&] {
        return launch_propose(v, MODE_EVAL, 0u, nullptr, x, n, uses_tc(v), rho, h->d_status, h->stream);
    });
    if (st != QST_OK) return st;
    st = enqueue_projection(h, *hp, n, p);
    if (st != QST_OK) return st;
    if (logl) {
        st = launch(h, QST_KERNEL_DIAG, "logl combine", [&] { return launch_logl_combine(v, n, logl, h->stream); });
        if (st != QST_OK) return st;
    }
    return QST_OK;
}

qst_status qst_set_profiling(qst_handle *h, int32_t enabled) {
    if (!h) return fail(QST_ERR_INVALID_ARG, "handle is NULL");
    h->prof = enabled != 0;
    return QST_OK;
}

qst_status qst_kernel_time(qst_handle *h, int32_t kind, int32_t reset, double *total_ms, int64_t *launches) {
    if (!h) return fail(QST_ERR_INVALID_ARG, "handle is NULL");
    if (kind < 0 || kind >= QST_KERNEL_KINDS) return fail(QST_ERR_INVALID_ARG, "unknown kernel kind");
    qst_status st = harvest(h);
    if (st != QST_OK) return st;
    if (total_ms) *total_ms = h->kind_ms[kind];
    if (launches) *launches = h->kind_launches[kind];
    if (reset) {
        for (int k = 0; k < QST_KERNEL_KINDS; ++k) {
            h->kind_ms[k] = 0.0;
            h->kind_launches[k] = 0;
        }
    }
    return QST_OK;
}

int64_t qst_launch_count(const qst_handle *h) { return h ? h->launches : 0; }

qst_status qst_philox_blocks(uint64_t seed, uint32_t step, uint32_t tag, uint32_t chain0, int64_t nchains,
                             uint32_t block0, int32_t nblocks, uint32_t *out, void *cuda_stream) {
    if (nchains < 0 || nblocks < 0 || (!out && nchains * nblocks > 0)) return fail(QST_ERR_INVALID_ARG, "bad sizes");
    cudaError_t e = launch_philox_blocks(seed, step, tag, chain0, nchains, block0, nblocks, out,
                                         reinterpret_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "philox");
    return QST_OK;
}

qst_status qst_pack_projectors(int32_t num_qubits, int32_t num_povms, const double *povm_re, const double *povm_im,
                               float *P_out) {
    if (num_qubits < 1 || num_qubits > 5 || num_povms < 1 || num_povms > kMaxPovmElements >> num_qubits || !povm_re ||
        !povm_im || !P_out)
        return fail(QST_ERR_INVALID_ARG, "bad arguments");
    const int D = 1 << num_qubits, KD = num_povms * D;
    std::vector<double> P((size_t)D * D * KD);
    pack_projectors(D, KD, povm_re, povm_im, P.data(), KD);
    for (size_t i = 0; i < P.size(); ++i) P_out[i] = (float)P[i];
    return QST_OK;
}

qst_status qst_pauli_povms(int32_t num_qubits, double *povm_re, double *povm_im) {
    if (num_qubits < 1 || num_qubits > 5) return fail(QST_ERR_INVALID_ARG, "num_qubits %d outside 1..5", num_qubits);
    if (!povm_re || !povm_im) return fail(QST_ERR_INVALID_ARG, "NULL output");
    std::vector<double> re, im;
    pauli_povms(num_qubits, re, im);
    std::memcpy(povm_re, re.data(), sizeof(double) * re.size());
    std::memcpy(povm_im, im.data(), sizeof(double) * im.size());
    return QST_OK;
}

qst_status qst_probe_wait_timeout(qst_handle *h, int32_t wait_ms) {
    if (!h) return fail(QST_ERR_INVALID_ARG, "NULL handle");
    if (wait_ms < 1 || wait_ms > 2000) return fail(QST_ERR_INVALID_ARG, "wait_ms must be in 1..2000");
    QST_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    uint32_t before = 0;
    QST_CUDA(cudaMemcpy(&before, h->d_status, sizeof(before), cudaMemcpyDeviceToHost), "read status");
    if (before != 0) return check_status(h);   // a real failure is pending: report it, clear nothing
    QST_CUDA(launch_wait_timeout_probe(h->d_status, (uint64_t)wait_ms * 1000000ull, h->stream), "probe launch");
    const qst_status st = check_status(h);
    const uint32_t zero = 0;
    QST_CUDA(cudaMemcpy(h->d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice), "clear status");
    return st;
}

qst_status qst_inject_nan(qst_handle *h, int32_t problem, int64_t chain) {
    HostProblem *hp;
    qst_status st = get_problem(h, problem, &hp);
    if (st != QST_OK) return st;
    if (chain < 0 || chain >= hp->v.R) return fail(QST_ERR_INVALID_ARG, "chain out of range");
    return launch(h, QST_KERNEL_DIAG, "inject nan", [&] { return launch_inject_nan(hp->v, chain, h->stream); });
}

}  // extern "C"
