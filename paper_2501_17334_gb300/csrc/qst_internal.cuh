// Internal definitions of the GB300 sampler: device-side problem view, kernel
// argument blocks, the counter-based generator and launch declarations.
#pragma once

#include "log_poly.h"
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace qst {

// Device status bits (read back by synchronising calls).
enum : uint32_t {
    STATUS_TIMEOUT = 1u << 0,     // a bounded mbarrier wait gave up
    STATUS_BOUNDS = 1u << 1,      // a kernel's own bounds check failed
    STATUS_BAD_LAUNCH = 1u << 2,  // a kernel was launched with an unsupported shape
};

// Stream tags of the counter layout (block, step j, global chain id, tag).
enum : uint32_t { TAG_INIT = 0, TAG_PROPOSAL = 1, TAG_ALPHA = 2 };

enum ProposeMode : int { MODE_INIT = 0, MODE_STEP = 1, MODE_EVAL = 2 };

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplications whose high halves are xored into the other two words with the
// round key, the key bumped by the Weyl constants after every round.
// ---------------------------------------------------------------------------------------
struct Philox {
    static constexpr uint32_t kMulA = 0xD2511F53u;
    static constexpr uint32_t kMulB = 0xCD9E8D57u;
    static constexpr uint32_t kWeylA = 0x9E3779B9u;
    static constexpr uint32_t kWeylB = 0xBB67AE85u;

    __device__ __forceinline__ static uint4 block(uint4 ctr, uint32_t key_lo, uint32_t key_hi) {
#pragma unroll
        for (int round = 0; round < 10; ++round) {
            const uint32_t pa_hi = __umulhi(kMulA, ctr.x);
            const uint32_t pa_lo = kMulA * ctr.x;
            const uint32_t pb_hi = __umulhi(kMulB, ctr.z);
            const uint32_t pb_lo = kMulB * ctr.z;
            ctr = make_uint4(pb_hi ^ ctr.y ^ key_lo, pb_lo, pa_hi ^ ctr.w ^ key_hi, pa_lo);
            key_lo += kWeylA;
            key_hi += kWeylB;
        }
        return ctr;
    }

    // The same block with the ten round keys (key + r (kWeylA, kWeylB)) given: a kernel that
    // takes them as launch parameters reads them as constant operands instead of forming them.
    struct RoundKeys {
        uint32_t k[20];   // (lo, hi) of rounds 0..9
    };
    __host__ __device__ static RoundKeys round_keys(uint64_t seed) {
        RoundKeys rk;
        uint32_t lo = (uint32_t)(seed & 0xffffffffu), hi = (uint32_t)(seed >> 32);
        for (int r = 0; r < 10; ++r) {
            rk.k[2 * r] = lo;
            rk.k[2 * r + 1] = hi;
            lo += kWeylA;
            hi += kWeylB;
        }
        return rk;
    }
    __device__ __forceinline__ static uint4 block(uint4 ctr, const RoundKeys &rk) {
#pragma unroll
        for (int round = 0; round < 10; ++round) {
            const uint32_t pa_hi = __umulhi(kMulA, ctr.x);
            const uint32_t pa_lo = kMulA * ctr.x;
            const uint32_t pb_hi = __umulhi(kMulB, ctr.z);
            const uint32_t pb_lo = kMulB * ctr.z;
            ctr = make_uint4(pb_hi ^ ctr.y ^ rk.k[2 * round], pb_lo, pa_hi ^ ctr.w ^ rk.k[2 * round + 1], pa_lo);
        }
        return ctr;
    }

    // Open-interval uniform from the top 23 bits m: (2 m + 1) 2^-24, exact in float.  Formed
    // by bit operations: 1 + m 2^-23 is the float with m as its mantissa, and subtracting
    // 1 - 2^-24 (a float) leaves (2 m + 1) 2^-24, representable, so the subtraction is exact.
    __device__ __forceinline__ static float uniform(uint32_t word) {
        return __int_as_float(0x3f800000u | (word >> 9)) - 0x1.fffffep-1f;
    }

    // Box-Muller on one uniform pair: (sqrt(-2 ln u) cos 2 pi v, sqrt(-2 ln u) sin 2 pi v).
    __device__ __forceinline__ static void gaussian_pair(uint32_t wu, uint32_t wv, float &z0, float &z1) {
        const float u = uniform(wu);
        const float v = uniform(wv);
        const float radius = sqrtf(-2.0f * logf(u));
        float s, c;
        sincospif(2.0f * v, &s, &c);
        z0 = radius * c;
        z1 = radius * s;
    }
};

// ---------------------------------------------------------------------------------------
// Device view of one problem.  Dimensions: D = 2^Q, d = D^2 (packed rho), nx = 4 D^2
// (latent), KD = K*D projectors, d_pad = d rounded up to 64 (operand rows), KD_pad =
// KD rounded up to the contraction's column tile.
// ---------------------------------------------------------------------------------------
// log x for the likelihood terms: the polynomial logarithm (log_poly.h, <= 1 ulp) for
// positive normal x; -inf when x <= 0 (or below the normal range), so a counted outcome
// with p <= 0 makes log L = -inf and the proposal is rejected.  (A NaN or infinite rho
// reaches log L through its trace instead.)
__device__ __forceinline__ float deviance_log(float x) {
    const float r = qst_log_poly(x);
    return (__float_as_int(x) >= 0x00800000) ? r : -INFINITY;
}

// Step counter kept on the device, so that a step's launches have fixed arguments and can
// be captured once in a CUDA graph: advance_step_kernel opens step j = step + 1 and decides
// whether it is kept (j % T == 0 and j > burn_in) and at which trajectory index.
struct StepState {
    uint32_t step;       // j of the step being run (0 before the first)
    int32_t kept;        // step j is kept
    int64_t kept_idx;    // index of step j's state among the kept states
    int64_t kept_count;  // kept states so far, this step included
};

// Operand kind of the tensor-core projection (the mixed forms).  TC_BF16X3: rho split into
// bf16 hi + mid + lo, P in bf16 (kind::f16).  TC_TF32: rho rounded to TF32 once, P in TF32
// (kind::tf32).  TC_TF32X2: rho = hi + lo, both TF32 (kind::tf32).
enum TcKind { TC_NONE = 0, TC_BF16X3 = 1, TC_TF32 = 2, TC_TF32X2 = 3 };
__host__ __device__ constexpr int tc_splits(int kind) { return kind == TC_BF16X3 ? 3 : kind == TC_TF32X2 ? 2 : 1; }
__host__ __device__ constexpr int tc_elem_bytes(int kind) { return kind == TC_BF16X3 ? 2 : 4; }

struct ProblemView {
    int D, d, nx, KD, KD_pad, d_pad;
    int tc_kind;                 // TcKind of the projection (TC_NONE: the plain FP32 form)
    int KD_tc;                   // columns of the tensor-core operand (multiple of its N tile)
    int64_t R;
    int64_t chain_offset;
    uint64_t seed;
    double C0;     // constant of the deviance form: -sum_{c>0} c log(invf), and for the Poisson
                   // likelihood + sum_{c>0} c log(mu_k) - sum_k mu_k (see the projection kernels)
    double Ntot;   // sum of all counts: weight of log t (trace of the stored rho) in log L
    int poisson;   // 0: the multinomial likelihood (Eq. likelihood); 1: Poisson counts of mean mu_k p_kl

    // packed projector operands and per-column likelihood weights
    const float *P32;            // [d_pad][KD_pad]  (row = packed rho index, contiguous columns)
    const void *Ptc;             // [KD_tc][d_pad]   tensor-core B operand (row = projector, contiguous packed
                                 //                  index): bf16, or FP32 holding TF32 values
    const float *cnt;            // [max(KD_pad, KD_tc)] counts as float, 0 on padding
    const float *invf;           // [max(KD_pad, KD_tc)] P_k / c_kl, Poisson: mu_k / c_kl (1 where c_kl = 0)
    const float *ptot;           // [max(KD_pad, KD_tc) / D] shots P_k of each setting, Poisson: its expected
                                 //                  trials mu_k (0 on padding)
    const float4 *colw;          // [max(KD_pad, KD_tc) / 2] per column pair (invf, invf, add, add), tensor epilogue
    int pauli;                   // the structured Pauli form of the projection (project_pauli.cu)
    const float4 *pauli_wq;      // [KD / 2] deviance weights per output pair in the structured form's order
    const float2 *pauli_wc;      // [KD / 2] and their counts (pauli_weights)
    const int32_t *pauli_perm;   // [KD] tree order -> setting-major projector index

    // chain state
    float *y;                    // [2][R][nx] double-buffered latent states
    uint8_t *cur;                // [R] which y buffer holds the current state
    float *rho_cur;              // [R][d_pad] packed rho of the current state
    float *rho_prop;             // [R][d_pad] packed rho of the proposal (FP32 operand)
    void *rho_split;             // [R][tc_splits][d_pad] the same split for the tensor cores: bf16 hi/mid/lo,
                                 //                  or FP32 TF32 hi[, lo]
    double *trace_prop;          // [R] exact FP64 sum of rho_prop's stored diagonal (1 up to rounding)
    double *logl_cur;            // [R]
    double *logl_part;           // [ngroups][R] partial deviance sums of the proposal
    double *beta;                // [R]
    float2 *coef;                // [R] (sqrt(1 - beta^2), beta) rounded to FP32, for the proposal
    int32_t *acc_win;            // [R] accepts in the current adaptation window
    int64_t *acc_total;          // [R]
    double *pool;                // [n_slots][d] FP64 pooled sums, one slot per accept CTA
    int n_slots;
    int accept_cpc;              // chains per accept CTA (n_slots = ceil(R / accept_cpc))
    float *traj;                 // [n_diag][traj_cap][d] kept states of the diagnostic chains
    int n_diag;
    int traj_cap;
    uint8_t *trace_acc;          // [trace_steps][R]
    double *trace_logl;          // [trace_steps][R]
    int trace_steps;
    int ngroups;                 // column groups of the projection (partial sums per group)
    int qr_passes;               // 1 or 2 modified Gram-Schmidt passes, 3: one pass and the refinement; 0: no QR
                                 // (Hilbert-Schmidt prior, W = G)
    int propose_threads = 128;   // CTA size of the proposal kernel at D <= 16 (32, 64 or 128; autotuned)
};

struct SamplerParams {
    int32_t adapt_interval;
    double acc_lo, acc_hi, adapt_factor, beta_max;
};

// ---------------------------------------------------------------------------------------
// Launchers (each returns the CUDA launch error).
// ---------------------------------------------------------------------------------------
cudaError_t launch_advance_step(StepState *st, int thin, int burn_in, cudaStream_t s);
// step_dev: when not null the step is read from it (MODE_STEP), else `step` is used
cudaError_t launch_propose(const ProblemView &p, int mode, uint32_t step, const StepState *step_dev, const float *x_eval, int64_t n_eval,
                           bool want_split, float *rho_norm_out, uint32_t *status, cudaStream_t s);
cudaError_t launch_project_fp32(const ProblemView &p, const float *A, int64_t rows, double *out_part,
                                float *p_out, cudaStream_t s);
cudaError_t launch_accept(const ProblemView &p, const SamplerParams &sp, int mode, const StepState *step_dev, uint32_t step, bool kept,
                          int64_t kept_idx, uint32_t *status, cudaStream_t s);
cudaError_t launch_pool_reduce(const ProblemView &p, double *out, cudaStream_t s);
cudaError_t launch_acf(const ProblemView &p, int n_kept, int lmax, double *acf_raw, cudaStream_t s);
cudaError_t launch_logl_combine(const ProblemView &p, int64_t rows, double *out, cudaStream_t s);
cudaError_t launch_philox_blocks(uint64_t seed, uint32_t step, uint32_t tag, uint32_t chain0, int64_t nchains,
                                 uint32_t block0, int32_t nblocks, uint32_t *out, cudaStream_t s);
cudaError_t launch_inject_nan(const ProblemView &p, int64_t chain, cudaStream_t s);

// tcgen05 projection in the view's tc_kind (sm_103a).  Returns cudaErrorNotSupported if the
// shape is outside what the kernel handles.
struct TcPlan;
cudaError_t tc_plan_create(const ProblemView &p, const void *A_split, int64_t rows, TcPlan **plan);
void tc_plan_destroy(TcPlan *plan);
cudaError_t launch_project_tc(const TcPlan *plan, const ProblemView &p, int64_t rows, double *out_part,
                              float *p_out, uint32_t *status, cudaStream_t s);
int tc_ngroups(const ProblemView &p, int64_t rows);
int tc_column_tile(int D, int KD);       // N tile of the tensor-core contraction for KD columns (0 = unsupported)
bool tc_supported(int kind, int D);      // the tensor-core kernels handle this operand kind at this D
// test hook: one bounded mbarrier wait that nothing satisfies (sets STATUS_TIMEOUT after limit_ns)
cudaError_t launch_wait_timeout_probe(uint32_t *status, uint64_t limit_ns, cudaStream_t s);
int fp32_ngroups(const ProblemView &p, int64_t rows);
// Structured Pauli form: log L partials [rows] (one column group) and optionally p [rows][KD].
cudaError_t launch_project_pauli(const ProblemView &p, const float *A, int64_t rows, double *out, float *p_out,
                                 cudaStream_t s);
void pauli_tree_order(int Q, std::vector<int32_t> &perm);   // perm[o] = k D + l of tree output o
// the structured form's per-pair weights from the setting-major counts and P_k / c
void pauli_weights(int Q, const std::vector<int32_t> &perm, const float *cnt, const float *invf,
                   std::vector<float4> &wq, std::vector<float2> &wc);
void set_last_error(const char *msg);   // message returned by qst_last_error()
// chains per accept CTA for R chains of d packed floats each (a power of two, 8..128)
int accept_chains_per_cta(int64_t R, int d);

}  // namespace qst
