// Mixed-precision projector contraction on the 5th-generation tensor cores (sm_103a)
// with the fused log-likelihood epilogue (Sec. II, p_kl = Tr Lambda_kl rho; Eq. likelihood).
//
// q = vec_h(rho) . P as a BF16 GEMM with FP32 accumulation: the Pauli projector matrix P
// is exact in bf16 (entries 0 or +-2^-m), and the FP32 packed rho is split exactly into
// rho = hi + mid + lo (three bf16 terms, 24 significant bits), so
//     q = hi . P + (mid . P + lo . P)
// is a tcgen05 GEMM with K = 3 d_pad and FP32 accumulation in tensor memory, into two
// accumulators.  Every product hi_i P_ki has at most 8 significant bits, so the hi
// accumulator sums them without rounding unless a term lies 2^16 below the running sum;
// the mid and lo products go to a second accumulator, 2^8 smaller, whose roundings are
// that much smaller too.  The epilogue adds the two: q carries one FP32 rounding instead
// of one per MMA (a single accumulator rounds, one-sidedly, at the scale of q after each
// of the 3 d_pad / 16 MMAs), which halves the log L error of the contraction.
// The same kernel runs the TF32 forms (kind::tf32, K8 per MMA): rho rounded once to TF32
// (one accumulator), or split hi + lo (two), every split of A in shared memory.
//
// Persistent CTAs (one per SM) loop over work units: a tile of 128 chains (M = 128) times a
// range of its 128-column N tiles.  Whole rounds of the grid take whole chain tiles; the
// tiles of the last, partial round are split into column groups so that it still covers
// the SMs (a uniform split would reload A in every round).
//   warp 0 (one lane)  TMA producer of P tiles (128 projectors x 64 K) through a 5-stage ring;
//   warp 1             allocates all 512 TMEM columns (the hi and the mid + lo FP32
//                      accumulators, 128 columns each, and two buffers for the lo split of
//                      A); one lane issues tcgen05.mma (M128 N128 K16) and commits;
//   warp 2 (one lane)  TMA producer of the hi and mid splits of the A tile (128 x 2 d_pad
//                      bf16, SWIZZLE_128B, resident while a unit's N tiles run), one barrier
//                      pair per 64-wide K chunk: the next unit's chunk is loaded as soon as
//                      the last MMAs reading it finish;
//   warps 3-18         epilogue, four warps per TMEM lane quadrant (warp w may only read
//                      lanes 32 (w mod 4) ..), each owning 32 of a tile's 128 columns and
//                      writing its own partial sum per chain:
//                      tcgen05.ld its slice of both accumulators (TMEM lane = chain),
//                      release them (the MMAs of the next tile start as soon as every
//                      epilogue warp holds its slice in registers), add them and form the
//                      log-likelihood of each measurement setting k (D consecutive
//                      columns, all in one thread):
//                        sum_l c_kl log(q_kl invf_kl) - P_k log(S_k / t),  S_k = sum_l q_kl,
//                      FP32 per tile, FP64 across tiles.  At the start of a unit the same
//                      warps copy the next unit's lo split from global memory into the idle
//                      TMEM buffer (tcgen05.st), where the lo-split MMAs read A.  Keeping a
//                      third of A out of shared memory leaves room for five P stages, enough to
//                      cover the L2 latency of the P tiles.
// Renormalising every setting by its own computed sum S_k (instead of the trace t) is exact
// for a complete POVM (sum_l Lambda_kl = I gives S_k = t in real arithmetic) and cancels any
// error common to a setting's outcomes -- in particular the one-sided rounding of the
// tensor cores' FP32 accumulation, which otherwise shifts every q_kl of a chain the same
// way and adds N * bias to log L.  S_k is summed exactly as a hi + lo pair (each q split at
// 2^-20).  The last N tile of a problem issues its MMAs with N = the columns it has left.
// Every mbarrier wait is bounded (1 s of %globaltimer): on expiry the kernel sets the
// status word's TIMEOUT bit, stops every role, drains its MMAs and TMA loads (bounded
// again), frees TMEM and returns.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "qst_internal.cuh"
#include "f32x2.cuh"

namespace qst {
namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 128;
constexpr int TC_KATOM = 64;                       // bf16 elements per 128-byte swizzle row
constexpr int TC_ATOM_BYTES = TC_M * 128;          // 16 KB: 128 rows x 128 B (64 bf16 or 32 TF32 of K)
constexpr int TC_BSTAGES = 5;
constexpr int TC_EPI_PER_QUAD = 4;                           // epilogue warps per lane quadrant
constexpr int TC_EPI_COLS = TC_N / TC_EPI_PER_QUAD;           // columns per epilogue warp (32)
constexpr int TC_FIRST_EPI = 3;                               // first epilogue warp
constexpr int TC_THREADS = (TC_FIRST_EPI + 4 * TC_EPI_PER_QUAD) * 32;   // 608
constexpr int TC_MAX_KCHUNK = 8;                              // d_pad <= 256 at 32 TF32 per atom
constexpr uint32_t TC_TMEM_COLS = 512;   // hi and mid + lo accumulators, 2 buffers of the lo split
constexpr uint32_t TC_REST_COL = TC_N;         // first column of the mid + lo accumulator
constexpr uint32_t TC_ALO_COL = 2 * TC_N;      // first column of the lo-split buffers
constexpr uint64_t TC_WAIT_NS = 1000000000ull;     // 1 s

// What each operand kind keeps where (TcKind): K elements per 128-byte atom row, the A splits
// resident in shared memory, whether a bf16 lo split goes through tensor memory, whether a
// second accumulator takes the smaller splits, and the A/B format of the instruction
// descriptor (BF16 = 1, TF32 = 2).
template <int KIND>
struct TcOps {
    static constexpr int katom = 128 / tc_elem_bytes(KIND);
    static constexpr int smem_splits = KIND == TC_TF32 ? 1 : 2;
    static constexpr bool lo_in_tmem = KIND == TC_BF16X3;
    static constexpr bool two_acc = KIND != TC_TF32;
    static constexpr uint32_t fmt = KIND == TC_BF16X3 ? 1u : 2u;
};

struct TcArgs {
    const void *a_split;   // [rows][splits d_pad] the A operand (bf16 hi, mid, lo -- lo through TMEM -- or TF32 hi[, lo])
    const float4 *colw;    // [KD_tc / 2] per column pair (invf, invf, add, add): x = q invf + add
    const float *cnt;      // [KD_tc] counts as float
    const float *ptot;     // [KD_tc / D] shots per setting
    const double *trace;   // [rows] exact trace of the stored rho
    double *out;           // [ngroups * 4][rows] partial sums (one per epilogue column slice)
    float *p_out;          // [rows][KD] or null
    uint32_t *status;
    int64_t rows;
    int64_t units;         // full_units + (M tiles - full_units) * ngroups
    int64_t full_units;    // the first full_units units are whole chain tiles (all N tiles)
    int KD;
    int n_katoms;          // d_pad / (K elements per atom)
    int ntiles;            // KD_tc / 128
    int tiles_per_group;
    int ngroups;
    int poisson;           // 1: each setting adds -mu_k (S_k / t - 1) (Poisson) instead of -P_k log(S_k / t)
};

// ---- PTX wrappers ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// One bounded try: the thread may be suspended until the phase completes or a system-dependent
// time limit passes.  (A suspend-time hint of 1 ms, tried first, woke the waiting warps later:
// the tensor-core kernel took 4% longer.)
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait, taken by a whole warp in lockstep: true when the phase of `parity` completed,
// false on abort or after about 1 s (then the status word's TIMEOUT bit is set and every role
// stops).  Every lane polls and the warp votes, so the loop and everything after it stay
// warp-uniform (values the issuing warps derive there can live in uniform registers).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort_flag, uint32_t *status,
                                               uint64_t limit_ns = TC_WAIT_NS) {
    uint64_t t0 = 0;
    for (uint32_t it = 0; it < (1u << 28); ++it) {
        if (__all_sync(0xffffffffu, mbar_try(bar, parity))) return true;
        if ((it & 31) == 31) {
            if (__any_sync(0xffffffffu, *abort_flag != 0)) return false;
            const uint64_t now = __shfl_sync(0xffffffffu, global_timer(), 0);
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit_ns) {
                break;
            }
        }
    }
    if ((threadIdx.x & 31) == 0) {
        *abort_flag = 1;
        atomicOr(status, STATUS_TIMEOUT);
    }
    return false;
}
// Wait used while draining after an abort: ignores the abort flag, still bounded.
__device__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = global_timer();
    for (uint32_t it = 0; it < (1u << 28); ++it) {
        if (mbar_try(bar, parity)) return;
        if ((it & 31) == 31 && global_timer() - t0 > TC_WAIT_NS) return;
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// UMMA shared-memory descriptor: K-major, SWIZZLE_128B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024u >> 4) << 32;               // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // SWIZZLE_128B
    return d;
}
// Instruction descriptor of kind::f16 (fmt 1: A/B BF16) and kind::tf32 (fmt 2: A/B TF32): D F32,
// both operands K-major, M = 128, N = n (a multiple of 16: the last N tile of a problem only
// covers its remaining columns).
__host__ __device__ constexpr uint32_t mma_idesc(int n, uint32_t fmt = 1u) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
// M128 Nn K8 TF32 MMA, both operands from shared memory (one 32-byte K step, as above)
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
template <int KIND>
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    if constexpr (KIND == TC_BF16X3)
        mma_bf16(d_tmem, a, b, idesc, accumulate);
    else
        mma_tf32(d_tmem, a, b, idesc, accumulate);
}
// the bf16 MMA with A read from tensor memory (row m = TMEM lane m, K packed two per column)
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// one lane of the (converged) warp: true in exactly one lane
__device__ __forceinline__ bool elect_one() {
    uint32_t pred;
    asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n" : "=r"(pred));
    return pred != 0;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t ta, float (&va)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) va[i] = __uint_as_float(r[i]);
}
// two 32-column slices (the same lanes), one wait for both
__device__ __forceinline__ void tmem_ld32_pair(uint32_t ta, uint32_t tb, float (&va)[32], float (&vb)[32]) {
    uint32_t r[32], q[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]), "=r"(q[8]),
          "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15]), "=r"(q[16]),
          "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]), "=r"(q[23]), "=r"(q[24]),
          "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        va[i] = __uint_as_float(r[i]);
        vb[i] = __uint_as_float(q[i]);
    }
}

// 32 lanes x NC columns of 32-bit words from registers into tensor memory
template <int NC>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t (&r)[NC]) {
    static_assert(NC == 4 || NC == 8 || NC == 32, "tmem_st: 4, 8 or 32 columns");
    if constexpr (NC == 4) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
                     "r"(r[2]), "r"(r[3])
                     : "memory");
    } else if constexpr (NC == 8) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                     "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                     : "memory");
    } else {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
            "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
            "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
            "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
            : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Padded K (d_pad) of the packed rho for D: D^2 rounded up to 64.
__host__ __device__ constexpr int tc_dpad(int D) { return (D * D + 63) / 64 * 64; }

// POISSON: the Poisson likelihood's setting term (a compile-time choice, so that the
// multinomial instantiation carries none of its code)
template <int D, int KIND, bool POISSON>
__global__ void __launch_bounds__(TC_THREADS, 1)
    project_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
    using T = TcOps<KIND>;
    extern __shared__ uint8_t dyn_smem[];
    __shared__ __align__(8) uint64_t bar_a_full[TC_MAX_KCHUNK];
    __shared__ __align__(8) uint64_t bar_a_empty[TC_MAX_KCHUNK];
    __shared__ __align__(8) uint64_t bar_b_full[TC_BSTAGES];
    __shared__ __align__(8) uint64_t bar_b_empty[TC_BSTAGES];
    __shared__ __align__(8) uint64_t bar_acc_full;
    __shared__ __align__(8) uint64_t bar_acc_empty;
    __shared__ __align__(8) uint64_t bar_alo_full[2];
    __shared__ __align__(8) uint64_t bar_mma_done;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;

    const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x / 32), 0);   // provably warp-uniform
    const int lane = threadIdx.x % 32;
    // 1024-byte aligned, by pointer arithmetic on the shared array (so accesses stay ld.shared)
    uint8_t *base = dyn_smem + ((1024u - (smem_u32(dyn_smem) & 1023u)) & 1023u);
    const int nk = a.n_katoms;
    uint8_t *smA = base;                                          // atom (split sp, chunk kc) at sp * nk + kc
    uint8_t *smB = base + (size_t)T::smem_splits * nk * TC_ATOM_BYTES;
    // the epilogue's per-column weights, staged once: (invf, invf, add, add) and (c, c) per column
    // pair, shots per setting
    const int kd_tc = a.ntiles * TC_N;
    float4 *w_q = reinterpret_cast<float4 *>(smB + (size_t)TC_BSTAGES * TC_ATOM_BYTES);
    float2 *w_c = reinterpret_cast<float2 *>(w_q + kd_tc / 2);
    float *w_p = reinterpret_cast<float *>(w_c + kd_tc / 2);
    for (int i = threadIdx.x; i < kd_tc / 2; i += blockDim.x) {
        w_q[i] = __ldg(a.colw + i);
        w_c[i] = __ldg(reinterpret_cast<const float2 *>(a.cnt) + i);
    }
    for (int i = threadIdx.x; i < kd_tc / D; i += blockDim.x) w_p[i] = __ldg(a.ptot + i);
    // Work unit u: the first full_units units (whole rounds of the grid) are whole chain tiles;
    // every later chain tile is split into ngroups units, each a balanced range of its N tiles
    // (never empty: ngroups <= ntiles), so the last round still occupies every SM.
    auto unit_mtile = [&](int64_t u) -> int64_t {
        return u < a.full_units ? u : a.full_units + (u - a.full_units) / a.ngroups;
    };
    auto unit_group = [&](int64_t u) -> int { return u < a.full_units ? 0 : (int)((u - a.full_units) % a.ngroups); };
    auto unit_tiles = [&](int64_t u, int &tb, int &te) {
        if (u < a.full_units) {
            tb = 0;
            te = a.ntiles;
            return;
        }
        const int g = unit_group(u);
        tb = g * a.ntiles / a.ngroups;
        te = (g + 1) * a.ntiles / a.ngroups;
    };
    // i-th tile a unit visits: its range rotated by the unit's chain tile, so the CTAs running
    // side by side read different P tiles from L2 instead of all the same lines at once
    auto tile_at = [&](int64_t u, int tb, int te, int i) {
        const int len = te - tb;
        int j = i + (int)(unit_mtile(u) % len);
        if (j >= len) j -= len;
        return tb + j;
    };

    if (threadIdx.x == 0) {
        for (int kc = 0; kc < TC_MAX_KCHUNK; ++kc) {
            mbar_init(smem_u32(&bar_a_full[kc]), 1);
            mbar_init(smem_u32(&bar_a_empty[kc]), 1);
        }
        for (int s = 0; s < TC_BSTAGES; ++s) {
            mbar_init(smem_u32(&bar_b_full[s]), 1);
            mbar_init(smem_u32(&bar_b_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_acc_full), 1);
        mbar_init(smem_u32(&bar_acc_empty), 4 * TC_EPI_PER_QUAD);   // one arrival per epilogue warp
        for (int s = 0; s < 2; ++s) mbar_init(smem_u32(&bar_alo_full[s]), 4 * TC_EPI_PER_QUAD);
        mbar_init(smem_u32(&bar_mma_done), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0) {
        // ---------------- P-tile producer (whole warp in lockstep, one lane issues) ----------------
        int it = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
            int tb, te;
            unit_tiles(u, tb, te);
            for (int i = 0; i < te - tb && ok; ++i) {
                const int t = tile_at(u, tb, te, i);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % TC_BSTAGES;
                    const uint32_t ph = (uint32_t)(it / TC_BSTAGES) & 1u;
                    if (!mbar_wait_warp(smem_u32(&bar_b_empty[s]), ph ^ 1u, &abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    if (elect_one()) {
                        mbar_expect_tx(smem_u32(&bar_b_full[s]), (uint32_t)TC_ATOM_BYTES);
                        tma_load_2d(smem_u32(smB + (size_t)s * TC_ATOM_BYTES), &tmB, kc * T::katom, t * TC_N,
                                    smem_u32(&bar_b_full[s]));
                    }
                    __syncwarp();
                }
            }
        }
        if (!ok && lane == 0) {
            // no copy may still be writing shared memory when the CTA exits
            for (int back = 1; back <= TC_BSTAGES && it - back >= 0; ++back) {
                const int i2 = it - back;
                mbar_drain(smem_u32(&bar_b_full[i2 % TC_BSTAGES]), (uint32_t)(i2 / TC_BSTAGES) & 1u);
            }
        }
    } else if (warp == 2) {
        // ---------------- A-tile producer (whole warp in lockstep, one lane issues) ----------------
        uint32_t uc = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
            int tb, te;
            unit_tiles(u, tb, te);
            if (te <= tb) continue;
            const int m0 = (int)(unit_mtile(u) * TC_M);
            for (int kc = 0; kc < nk; ++kc) {
                if (!mbar_wait_warp(smem_u32(&bar_a_empty[kc]), (uc & 1u) ^ 1u, &abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                if (elect_one()) {
                    mbar_expect_tx(smem_u32(&bar_a_full[kc]), (uint32_t)(T::smem_splits * TC_ATOM_BYTES));
                    for (int sp = 0; sp < T::smem_splits; ++sp)
                        tma_load_2d(smem_u32(smA + (size_t)(sp * nk + kc) * TC_ATOM_BYTES), &tmA,
                                    (sp * nk + kc) * T::katom, m0, smem_u32(&bar_a_full[kc]));
                }
                __syncwarp();
            }
            ++uc;
        }
        if (!ok && lane == 0) {
            // the last unit's chunks that were issued
            for (int kc = 0; kc < nk; ++kc) mbar_drain(smem_u32(&bar_a_full[kc]), uc & 1u);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        // The whole warp runs the loop (so the descriptors are warp-uniform values); lane 0 issues
        // the MMAs and commits.  Descriptors advance by (byte offset >> 4) in their start field.
        int it = 0, tcount = 0;
        uint32_t uc = 0;
        bool ok = true;
        const uint64_t adesc0 = sw128_desc(smem_u32(smA)), bdesc0 = sw128_desc(smem_u32(smB));
        auto wait_all = [&](uint32_t bar, uint32_t parity) {
            return mbar_wait_warp(bar, parity, &abort_flag, a.status);
        };
        for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
            int tb, te;
            unit_tiles(u, tb, te);
            for (int i = 0; i < te - tb && ok; ++i, ++tcount) {
                const int t = tile_at(u, tb, te, i);
                const uint32_t use = (uint32_t)tcount & 1u;   // the accumulators' use parity
                if (!wait_all(smem_u32(&bar_acc_empty), use ^ 1u) ||
                    (T::lo_in_tmem && i == 0 && !wait_all(smem_u32(&bar_alo_full[uc & 1u]), (uc >> 1) & 1u))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_hi = tmem, d_rest = tmem + TC_REST_COL;
                const int n_valid = min(TC_N, (a.KD - t * TC_N + 15) / 16 * 16);
                const uint32_t idesc = mma_idesc(n_valid, T::fmt);
                const uint32_t alo_tmem = tmem + TC_ALO_COL + (uc & 1u) * (uint32_t)TC_N;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % TC_BSTAGES;
                    const uint32_t ph = (uint32_t)(it / TC_BSTAGES) & 1u;
                    if (!wait_all(smem_u32(&bar_b_full[s]), ph) ||
                        (i == 0 && !wait_all(smem_u32(&bar_a_full[kc]), uc & 1u))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t bd = bdesc0 + (uint64_t)((s * TC_ATOM_BYTES) >> 4);
                    const uint64_t ad_hi = adesc0 + (uint64_t)((kc * TC_ATOM_BYTES) >> 4);
                    const uint64_t ad_2 = adesc0 + (uint64_t)(((nk + kc) * TC_ATOM_BYTES) >> 4);   // mid / TF32 lo
                    const uint32_t ad_lo = alo_tmem + (uint32_t)(kc * TC_KATOM / 2);
                    if (elect_one()) {
                        // four MMAs per 128-byte atom row: 32 bytes of K (16 bf16 or 8 TF32) each,
                        // 2 descriptor units
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_ss<KIND>(d_hi, ad_hi + 2 * kk, bd + 2 * kk, idesc, (kc | kk) != 0 ? 1u : 0u);
                        if constexpr (T::smem_splits == 2) {
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                mma_ss<KIND>(d_rest, ad_2 + 2 * kk, bd + 2 * kk, idesc, (kc | kk) != 0 ? 1u : 0u);
                        }
                        if constexpr (T::lo_in_tmem) {
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)   // lo split, A from tensor memory
                                mma_bf16_ta(d_rest, ad_lo + (uint32_t)(kk * 8), bd + 2 * kk, idesc, 1u);
                        }
                        mma_commit(smem_u32(&bar_b_empty[s]));
                        if (i == te - tb - 1) mma_commit(smem_u32(&bar_a_empty[kc]));   // last reader of this A chunk
                    }
                    __syncwarp();
                }
                if (!ok) break;
                if (elect_one()) mma_commit(smem_u32(&bar_acc_full));
                __syncwarp();
            }
            ++uc;
        }
        if (!ok && lane == 0) {
            // every MMA issued so far must finish before TMEM and shared memory go away
            mma_commit(smem_u32(&bar_mma_done));
            mbar_drain(smem_u32(&bar_mma_done), 0u);
        }
        __syncwarp();
    } else if (warp >= TC_FIRST_EPI) {
        // ---------------- epilogue ----------------
        const int quad = warp & 3;                        // TMEM lane quadrant this warp may access
        const int sub = (warp - TC_FIRST_EPI) / 4;        // column slice of every tile
        const int col0 = sub * TC_EPI_COLS;
        // The lo split of a unit's A rows goes from global memory into TMEM buffer b (the MMAs
        // read it there): this warp writes lanes 32 quad.., K elements [sub DP/4, (sub+1) DP/4).
        constexpr int DP = tc_dpad(D);
        constexpr int NCW = DP / 2 / TC_EPI_PER_QUAD;   // 32-bit TMEM columns per warp
        // It moves in pieces of 4 columns (16 bytes of each row): the next unit's pieces are
        // fetched one per tile at the start of the tile and stored at its end, so the global
        // loads never stall the epilogue.
        constexpr int NP = NCW / 4;
        auto alo_fetch = [&](int64_t u, int piece) {
            const int64_t row = unit_mtile(u) * TC_M + quad * 32 + lane;
            if (row >= a.rows) return make_uint4(0u, 0u, 0u, 0u);
            const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(a.a_split) +
                                                               row * 3 * DP + 2 * DP + sub * (DP / TC_EPI_PER_QUAD));
            return __ldg(src + piece);
        };
        auto alo_store = [&](uint32_t b, int piece, uint4 w) {
            const uint32_t r[4] = {w.x, w.y, w.z, w.w};
            tmem_st<4>(tmem + ((uint32_t)(quad * 32) << 16) + TC_ALO_COL + b * (uint32_t)TC_N +
                           (uint32_t)(sub * NCW + 4 * piece),
                       r);
        };
        auto alo_done = [&](uint32_t b) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_alo_full[b]));
        };
        if (T::lo_in_tmem && blockIdx.x < a.units) {
            for (int piece = 0; piece < NP; ++piece) alo_store(0u, piece, alo_fetch(blockIdx.x, piece));
            alo_done(0u);
        }
        int tcount = 0;
        uint32_t ucount = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x, ++ucount) {
            // the next unit's lo split goes into the other buffer: its last readers (the MMAs of
            // the unit before this one) completed before this warp received that unit's last
            // accumulator
            const bool has_next = T::lo_in_tmem && u + gridDim.x < a.units;
            const uint32_t nb_buf = (ucount + 1) & 1u;
            int tb, te;
            unit_tiles(u, tb, te);
            const int g = unit_group(u);
            const int64_t grow = unit_mtile(u) * TC_M + quad * 32 + lane;
            const bool valid = grow < a.rows;
            // t = t_hi + t_lo exactly (an FP64 sum of FP32 values, a few ulps from 1); 1 / t in FP32
            // (it scales rel, itself a few ulps, and p), so the unit's FP64 work is these two
            // conversions and the final sum: on this part an FP64 instruction is scarce
            const double t = valid ? a.trace[grow] : 1.0;
            const float t_hi = (float)t;
            const float t_lo = (float)(t - (double)t_hi);
            const float inv_t = 1.0f / t_hi;
            float tot_hi = 0.0f, tot_lo = 0.0f;   // the unit's tile sums as an FP32 pair (two-sum)
            bool neg_inf = false;
            for (int i = 0; i < te - tb; ++i, ++tcount) {
                const int tt = tile_at(u, tb, te, i);
                const uint4 piece_w = (has_next && i < NP) ? alo_fetch(u + gridDim.x, i) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t use = (uint32_t)tcount & 1u;
                if (!mbar_wait_warp(smem_u32(&bar_acc_full), use, &abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int n0 = tt * TC_N + col0;
                float v[32];
                const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col0;
                if constexpr (T::two_acc) {
                    float vr[32];
                    tmem_ld32_pair(lane_base, lane_base + TC_REST_COL, v, vr);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty));   // the warp's slices are in registers
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const float2 q = add2(make_float2(v[i], v[i + 1]), make_float2(vr[i], vr[i + 1]));
                        v[i] = q.x;
                        v[i + 1] = q.y;
                    }
                } else {
                    tmem_ld32(lane_base, v);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty));   // the warp's slice is in registers
                }
                bool tile_neg_inf = false;
                if (n0 < a.KD) {   // (columns past KD: the last tile's MMA did not write them)
                    int xmin = 0x7fffffff;   // smallest bit pattern of a log argument (sign included)
#pragma unroll
                    for (int sk = 0; sk < TC_EPI_COLS / D; ++sk) {
                        const int nb = n0 + sk * D;               // first column of setting nb / D
                        const float pk = w_p[nb / D];
                        if (pk > 0.0f) {
                            // S_k = sum_l q_kl exactly as hi + lo: every q in (-4, 4) is split at
                            // 2^-20 by adding and removing 12 (so the hi parts add exactly), the
                            // lo parts are below 2^-21
                            float2 sh = splat2(0.0f), sl = splat2(0.0f), dev = splat2(0.0f), comp = splat2(0.0f);
                            float4 w_next = w_q[nb / 2];
                            float2 c_next = w_c[nb / 2];
#pragma unroll
                            for (int l = 0; l < D; l += 2) {
                                const float4 w = w_next;   // this pair's weights, the next pair's requested now
                                const float2 c = c_next;
                                if (l + 2 < D) {
                                    w_next = w_q[(nb + l + 2) / 2];
                                    c_next = w_c[(nb + l + 2) / 2];
                                }
                                const float2 q = make_float2(v[sk * D + l], v[sk * D + l + 1]);
                                const float2 h = sub2(add2(q, splat2(12.0f)), splat2(12.0f));
                                sh = add2(sh, h);
                                sl = add2(sl, sub2(q, h));
                                // deviance terms c log(q invf); columns without counts get x = 1
                                const float2 x = fma2(q, make_float2(w.x, w.y), make_float2(w.z, w.w));
                                xmin = min(xmin, min(__float_as_int(x.x), __float_as_int(x.y)));
                                kahan_fma2(dev, comp, c, log_poly2(x));
                            }
                            const float s_hi = sh.x + sh.y, s_lo = sl.x + sl.y;   // (s_hi exact)
                            if constexpr (POISSON) {
                                float ph, pl;
                                poisson_setting(pk, s_hi, s_lo, t_hi, t_lo, ph, pl);
                                add_setting_pair(tot_hi, tot_lo, dev, comp, ph, pl);
                            } else {
                                // log(S_k / t), S_k - t formed from the exact pairs (Sterbenz: s_hi - t_hi exact)
                                const float rel = ((s_hi - t_hi) + (s_lo - t_lo)) * inv_t;
                                // log1p(rel): |rel| is a few ulps, where three terms are exact to 2^-40
                                const float l1p = fabsf(rel) < 0x1p-10f
                                                      ? rel * __fmaf_rn(rel, __fmaf_rn(rel, 0.33333334f, -0.5f), 1.0f)
                                                      : log1pf(rel);
                                // the setting's term goes straight into the unit's pair
                                add_setting(tot_hi, tot_lo, dev, comp, pk * l1p);
                            }
                        }
                    }
                    // a counted outcome with q <= 0 (or below the normal range): log L = -inf
                    if (xmin < 0x00800000) tile_neg_inf = true;
                    if (a.p_out && valid) {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (n0 + i < a.KD) a.p_out[grow * a.KD + n0 + i] = v[i] * inv_t;
                    }
                }
                if (tile_neg_inf) neg_inf = true;
                if (has_next) {
                    if (i < NP) alo_store(nb_buf, i, piece_w);
                    if (i == te - tb - 1) {   // last tile of the unit: whatever is left, then publish
                        for (int piece = i + 1; piece < NP; ++piece)
                            alo_store(nb_buf, piece, alo_fetch(u + gridDim.x, piece));
                        alo_done(nb_buf);
                    }
                }
            }
            if (ok && valid) {
                a.out[(int64_t)(g * 4 + sub) * a.rows + grow] = neg_inf ? -INFINITY : (double)tot_hi + (double)tot_lo;
                if (u < a.full_units)   // a whole chain tile: its other groups' partials are zero
                    for (int g2 = 1; g2 < a.ngroups; ++g2) a.out[(int64_t)(g2 * 4 + sub) * a.rows + grow] = 0.0;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

// ---- five qubits (D = 32): A streamed with every N tile ------------------------------------
// A 128-chain tile of A is 3 x 1024 bf16 per chain (768 KB), more than an SM holds, so here a
// work unit is one (chain tile, N tile) pair and A's K chunks are streamed with P's through a
// 2-stage ring: stage = one 64-wide K chunk of A's hi, mid and lo splits (3 x 16 KB) and of
// the P tile (256 projectors x 64 = 32 KB).  N tiles are 256 wide (M128 N256 K16 MMAs, both
// operands from shared memory); TMEM holds the hi and the mid + lo accumulators, 256 columns
// each, as above.  The epilogue is the one above, on 64-column slices, with the weights read
// through L1 (they do not fit beside the ring).
constexpr int TCW_N = 256;
constexpr int TCW_STAGES = 2;
constexpr int TCW_STAGE_BYTES = 3 * TC_ATOM_BYTES + TCW_N * TC_KATOM * 2;   // 80 KB
constexpr int TCW_EPI_COLS = TCW_N / TC_EPI_PER_QUAD;                        // 64

template <bool POISSON>
__global__ void __launch_bounds__(TC_THREADS, 1)
    project_tc_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
    constexpr int D = 32;
    extern __shared__ uint8_t dyn_smem[];
    __shared__ __align__(8) uint64_t bar_full[TCW_STAGES];
    __shared__ __align__(8) uint64_t bar_empty[TCW_STAGES];
    __shared__ __align__(8) uint64_t bar_acc_full;
    __shared__ __align__(8) uint64_t bar_acc_empty;
    __shared__ __align__(8) uint64_t bar_mma_done;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;

    const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x / 32), 0);
    const int lane = threadIdx.x % 32;
    // 1024-byte aligned, by pointer arithmetic on the shared array (so accesses stay ld.shared)
    uint8_t *base = dyn_smem + ((1024u - (smem_u32(dyn_smem) & 1023u)) & 1023u);
    const int nk = a.n_katoms;   // 16 K chunks per split
    // unit u: chain tile u / ntiles, N tile u % ntiles
    if (threadIdx.x == 0) {
        for (int s = 0; s < TCW_STAGES; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_acc_full), 1);
        mbar_init(smem_u32(&bar_acc_empty), 4 * TC_EPI_PER_QUAD);   // one arrival per epilogue warp
        mbar_init(smem_u32(&bar_mma_done), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(2 * TCW_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0) {
        // ---------------- producer of A and P chunks ----------------
        int it = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
            const int m0 = (int)((u / a.ntiles) * TC_M);
            const int t = (int)(u % a.ntiles);
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = it % TCW_STAGES;
                const uint32_t ph = (uint32_t)(it / TCW_STAGES) & 1u;
                if (!mbar_wait_warp(smem_u32(&bar_empty[s]), ph ^ 1u, &abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                if (elect_one()) {
                    uint8_t *st = base + (size_t)s * TCW_STAGE_BYTES;
                    mbar_expect_tx(smem_u32(&bar_full[s]), (uint32_t)TCW_STAGE_BYTES);
                    for (int sp = 0; sp < 3; ++sp)
                        tma_load_2d(smem_u32(st + (size_t)sp * TC_ATOM_BYTES), &tmA, (sp * nk + kc) * TC_KATOM, m0,
                                    smem_u32(&bar_full[s]));
                    tma_load_2d(smem_u32(st + 3 * TC_ATOM_BYTES), &tmB, kc * TC_KATOM, t * TCW_N, smem_u32(&bar_full[s]));
                }
                __syncwarp();
            }
        }
        if (!ok && lane == 0) {
            for (int back = 1; back <= TCW_STAGES && it - back >= 0; ++back) {
                const int i2 = it - back;
                mbar_drain(smem_u32(&bar_full[i2 % TCW_STAGES]), (uint32_t)(i2 / TCW_STAGES) & 1u);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        int it = 0, tcount = 0;
        bool ok = true;
        const uint64_t desc0 = sw128_desc(smem_u32(base));
        for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x, ++tcount) {
            const int t = (int)(u % a.ntiles);
            const uint32_t use = (uint32_t)tcount & 1u;
            if (!mbar_wait_warp(smem_u32(&bar_acc_empty), use ^ 1u, &abort_flag, a.status)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t d_hi = tmem, d_rest = tmem + (uint32_t)TCW_N;
            const int n_valid = min(TCW_N, (a.KD - t * TCW_N + 15) / 16 * 16);
            const uint32_t idesc = mma_idesc(n_valid);
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = it % TCW_STAGES;
                const uint32_t ph = (uint32_t)(it / TCW_STAGES) & 1u;
                if (!mbar_wait_warp(smem_u32(&bar_full[s]), ph, &abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t sd = desc0 + (uint64_t)(((size_t)s * TCW_STAGE_BYTES) >> 4);
                const uint64_t bd = sd + (uint64_t)((3 * TC_ATOM_BYTES) >> 4);
                if (elect_one()) {
#pragma unroll
                    for (int sp = 0; sp < 3; ++sp) {   // hi into d_hi, mid and lo into d_rest
#pragma unroll
                        for (int kk = 0; kk < TC_KATOM / 16; ++kk)
                            mma_bf16(sp == 0 ? d_hi : d_rest, sd + (uint64_t)((sp * TC_ATOM_BYTES) >> 4) + 2 * kk,
                                     bd + 2 * kk, idesc, (kc | (sp >> 1) | kk) != 0 ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&bar_empty[s]));
                }
                __syncwarp();
            }
            if (!ok) break;
            if (elect_one()) mma_commit(smem_u32(&bar_acc_full));
            __syncwarp();
        }
        if (!ok && lane == 0) {
            mma_commit(smem_u32(&bar_mma_done));
            mbar_drain(smem_u32(&bar_mma_done), 0u);
        }
        __syncwarp();
    } else if (warp >= TC_FIRST_EPI) {
        // ---------------- epilogue (64-column slices) ----------------
        const int quad = warp & 3;
        const int sub = (warp - TC_FIRST_EPI) / 4;
        const int col0 = sub * TCW_EPI_COLS;
        int tcount = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x, ++tcount) {
            const int t = (int)(u % a.ntiles);
            const int64_t grow = (u / a.ntiles) * TC_M + quad * 32 + lane;
            const bool valid = grow < a.rows;
            const double tr = valid ? a.trace[grow] : 1.0;
            const float t_hi = (float)tr;
            const float t_lo = (float)(tr - (double)t_hi);
            const float inv_t = 1.0f / t_hi;
            const uint32_t use = (uint32_t)tcount & 1u;
            if (!mbar_wait_warp(smem_u32(&bar_acc_full), use, &abort_flag, a.status)) {
                ok = false;
                break;
            }
            tc_fence_after();
            float tile_hi = 0.0f, tile_lo = 0.0f;   // the tile's settings, summed as a pair
            int xmin = 0x7fffffff;
            float vv[2][32];   // q of this warp's two 32-column settings: hi + (mid + lo)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float vr[32];
                const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(col0 + 32 * half);
                tmem_ld32_pair(ta, ta + (uint32_t)TCW_N, vv[half], vr);
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float2 q = add2(make_float2(vv[half][i], vv[half][i + 1]), make_float2(vr[i], vr[i + 1]));
                    vv[half][i] = q.x;
                    vv[half][i + 1] = q.y;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty));   // the warp's slices are in registers
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int n0 = t * TCW_N + col0 + 32 * half;   // one setting of 32 outcomes
                const float *v = vv[half];
                if (n0 >= a.KD) continue;
                const float pk = __ldg(a.ptot + n0 / D);
                if (pk > 0.0f) {
                    float2 sh = splat2(0.0f), sl = splat2(0.0f), dev = splat2(0.0f), comp = splat2(0.0f);
#pragma unroll
                    for (int l = 0; l < D; l += 2) {
                        const float2 q = make_float2(v[l], v[l + 1]);
                        const float2 h = sub2(add2(q, splat2(12.0f)), splat2(12.0f));
                        sh = add2(sh, h);
                        sl = add2(sl, sub2(q, h));
                        const float4 w = __ldg(a.colw + (n0 + l) / 2);
                        const float2 c = __ldg(reinterpret_cast<const float2 *>(a.cnt + n0 + l));
                        const float2 x = fma2(q, make_float2(w.x, w.y), make_float2(w.z, w.w));
                        xmin = min(xmin, min(__float_as_int(x.x), __float_as_int(x.y)));
                        kahan_fma2(dev, comp, c, log_poly2(x));
                    }
                    const float s_hi = sh.x + sh.y, s_lo = sl.x + sl.y;
                    if constexpr (POISSON) {
                        float ph, pl;
                        poisson_setting(pk, s_hi, s_lo, t_hi, t_lo, ph, pl);
                        add_setting_pair(tile_hi, tile_lo, dev, comp, ph, pl);
                    } else {
                        const float rel = ((s_hi - t_hi) + (s_lo - t_lo)) * inv_t;
                        const float l1p = fabsf(rel) < 0x1p-10f
                                              ? rel * __fmaf_rn(rel, __fmaf_rn(rel, 0.33333334f, -0.5f), 1.0f)
                                              : log1pf(rel);
                        add_setting(tile_hi, tile_lo, dev, comp, pk * l1p);
                    }
                }
                if (a.p_out && valid) {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (n0 + i < a.KD) a.p_out[grow * a.KD + n0 + i] = v[i] * inv_t;
                }
            }
            if (valid)
                a.out[(int64_t)(t * 4 + sub) * a.rows + grow] =
                    xmin < 0x00800000 ? -INFINITY : (double)tile_hi + (double)tile_lo;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TCW_N));
    }
}

// Test hook for the failure path: one warp waits, through the same bounded wait as the kernels
// above, on an mbarrier that nothing ever arrives on.  After limit_ns the wait gives up, sets
// the status word's TIMEOUT bit and returns, and the kernel exits with nothing in flight.
__global__ void wait_timeout_probe_kernel(uint32_t *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    mbar_wait_warp(smem_u32(&bar), 0u, &abort_flag, status, limit_ns);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D row-major map (inner elements contiguous) of bf16 or FP32 elements, 128-byte swizzle
bool encode_2d(CUtensorMap *map, const void *ptr, int elem_bytes, uint64_t inner, uint64_t outer, uint32_t box_inner,
               uint32_t box_outer) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(map, dt, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// A (the splits held in shared memory), the P ring, then the epilogue's weights
size_t tc_smem_bytes(int kind, int n_katoms, int kd_tc, int D) {
    const int splits = kind == TC_TF32 ? 1 : 2;
    return 1024 + (size_t)(splits * n_katoms + TC_BSTAGES) * TC_ATOM_BYTES +
           (size_t)(kd_tc / 2) * (sizeof(float4) + sizeof(float2)) + (size_t)(kd_tc / D) * sizeof(float);
}

}  // namespace

struct TcPlan {
    CUtensorMap a;
    CUtensorMap b;
    const void *a_split;
    int kind;
    int n_katoms;
    int ntiles;
};

namespace {
template <int D, int KIND, bool POISSON>
cudaError_t launch_tc_dkp(const TcPlan *plan, const TcArgs &a, dim3 grid, size_t smem, cudaStream_t s) {
    static size_t attr_bytes = 0;
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(project_tc_kernel<D, KIND, POISSON>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    project_tc_kernel<D, KIND, POISSON><<<grid, TC_THREADS, smem, s>>>(plan->a, plan->b, a);
    return cudaGetLastError();
}
template <int D, int KIND>
cudaError_t launch_tc_dk(const TcPlan *plan, const TcArgs &a, dim3 grid, size_t smem, cudaStream_t s) {
    return a.poisson ? launch_tc_dkp<D, KIND, true>(plan, a, grid, smem, s)
                     : launch_tc_dkp<D, KIND, false>(plan, a, grid, smem, s);
}
template <bool POISSON>
cudaError_t launch_tc_wide(const TcPlan *plan, const TcArgs &a, dim3 grid, size_t smem, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(project_tc_wide_kernel<POISSON>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    project_tc_wide_kernel<POISSON><<<grid, TC_THREADS, smem, s>>>(plan->a, plan->b, a);
    return cudaGetLastError();
}
template <int D>
cudaError_t launch_tc_d(const TcPlan *plan, const TcArgs &a, dim3 grid, size_t smem, cudaStream_t s) {
    switch (plan->kind) {
        case TC_BF16X3: return launch_tc_dk<D, TC_BF16X3>(plan, a, grid, smem, s);
        case TC_TF32: return launch_tc_dk<D, TC_TF32>(plan, a, grid, smem, s);
        case TC_TF32X2:
            if constexpr (D <= 8) return launch_tc_dk<D, TC_TF32X2>(plan, a, grid, smem, s);
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}
}  // namespace

int tc_column_tile(int D, int KD) { return KD > 0 ? (D == 32 ? TCW_N : TC_N) : 0; }

cudaError_t launch_wait_timeout_probe(uint32_t *status, uint64_t limit_ns, cudaStream_t s) {
    wait_timeout_probe_kernel<<<1, 32, 0, s>>>(status, limit_ns);
    return cudaGetLastError();
}

// BF16x3 to D = 32 (the streamed kernel above D = 16); TF32 keeps its one A split in shared
// memory to D = 16 (128 KB at D = 16); TF32x2 keeps two, to D = 8.
bool tc_supported(int kind, int D) {
    switch (kind) {
        case TC_BF16X3: return D >= 2 && D <= 32;
        case TC_TF32: return D >= 2 && D <= 16;
        case TC_TF32X2: return D >= 2 && D <= 8;
        default: return false;
    }
}
// (a setting's D outcome columns never straddle a tile: D divides the tile width)

// Partial sums per chain: four column slices times the column groups that split the N tiles
// when there are too few chain tiles to occupy every SM.
int tc_ngroups(const ProblemView &p, int64_t rows) {
    if (p.D == 32) return 4 * (p.KD_tc / TCW_N);   // one partial per N tile and column slice
    const int64_t mt = (rows + TC_M - 1) / TC_M;
    const int ntiles = p.KD_tc / TC_N;
    int g = 1;
    if (mt >= 152) {   // whole rounds run undivided (tc_full_units); split the last round's tiles
        const int64_t rem = mt % 152;
        if (rem > 0) g = (int)std::min<int64_t>(ntiles, std::max<int64_t>(1, 152 / rem));
        return 4 * g;
    }
    while (g < ntiles && mt * g < 152) g *= 2;
    return 4 * (g > ntiles ? ntiles : g);
}

cudaError_t tc_plan_create(const ProblemView &p, const void *A_split, int64_t rows, TcPlan **plan) {
    *plan = nullptr;
    const int kind = p.tc_kind;
    if (!tc_supported(kind, p.D)) return cudaErrorNotSupported;
    const bool wide = p.D == 32;   // BF16x3 only
    const int n_tile = wide ? TCW_N : TC_N;
    const int eb = tc_elem_bytes(kind);
    const int katom = 128 / eb;
    if (p.d_pad % katom != 0 || p.KD_tc % n_tile != 0 || p.KD_tc <= 0) return cudaErrorNotSupported;
    const int n_katoms = p.d_pad / katom;
    if (!wide && n_katoms > TC_MAX_KCHUNK) return cudaErrorNotSupported;
    if (p.d_pad != tc_dpad(p.D)) return cudaErrorNotSupported;
    if (!wide && tc_smem_bytes(kind, n_katoms, p.KD_tc, p.D) > 227 * 1024 - 256) return cudaErrorNotSupported;
    if (reinterpret_cast<uintptr_t>(A_split) % 16 != 0 || reinterpret_cast<uintptr_t>(p.Ptc) % 16 != 0)
        return cudaErrorMisalignedAddress;
    TcPlan *pl = new TcPlan();
    pl->kind = kind;
    pl->n_katoms = n_katoms;
    pl->a_split = A_split;
    pl->ntiles = p.KD_tc / n_tile;
    const bool ok_a = encode_2d(&pl->a, A_split, eb, (uint64_t)tc_splits(kind) * p.d_pad, (uint64_t)rows, katom, TC_M);
    const bool ok_b = encode_2d(&pl->b, p.Ptc, eb, (uint64_t)p.d_pad, (uint64_t)p.KD_tc, katom, n_tile);
    if (!ok_a || !ok_b) {
        delete pl;
        return cudaErrorInvalidValue;
    }
    *plan = pl;
    return cudaSuccess;
}

void tc_plan_destroy(TcPlan *plan) { delete plan; }

cudaError_t launch_project_tc(const TcPlan *plan, const ProblemView &p, int64_t rows, double *out_part, float *p_out,
                              uint32_t *status, cudaStream_t s) {
    if (!plan) return cudaErrorInvalidValue;
    if (rows <= 0) return cudaSuccess;
    TcArgs a;
    a.a_split = plan->a_split;
    a.colw = p.colw;
    a.cnt = p.cnt;
    a.ptot = p.ptot;
    a.trace = p.trace_prop;
    a.out = out_part;
    a.p_out = p_out;
    a.status = status;
    a.rows = rows;
    a.KD = p.KD;
    a.n_katoms = plan->n_katoms;
    a.ntiles = plan->ntiles;
    a.poisson = p.poisson;
    const int groups = p.ngroups / 4;   // the epilogue writes four column-slice partials per group
    a.ngroups = groups;
    a.tiles_per_group = (plan->ntiles + groups - 1) / groups;
    static int num_sms = 0;
    if (num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms <= 0)
            num_sms = 148;
    }
    const int64_t mtiles = (rows + TC_M - 1) / TC_M;
    // whole rounds of the grid take whole chain tiles; the rest are split into `groups` units
    a.full_units = (p.D == 32) ? 0 : (mtiles / num_sms) * num_sms;
    a.units = (p.D == 32) ? mtiles * groups : a.full_units + (mtiles - a.full_units) * groups;
    dim3 grid((unsigned)std::min<int64_t>(a.units, num_sms));
    if (p.D == 32) {   // units: (chain tile, N tile) pairs
        const size_t smem = 1024 + (size_t)TCW_STAGES * TCW_STAGE_BYTES;
        return a.poisson ? launch_tc_wide<true>(plan, a, grid, smem, s) : launch_tc_wide<false>(plan, a, grid, smem, s);
    }
    const size_t smem = tc_smem_bytes(plan->kind, plan->n_katoms, plan->ntiles * TC_N, p.D);
    switch (p.D) {
        case 2: return launch_tc_d<2>(plan, a, grid, smem, s);
        case 4: return launch_tc_d<4>(plan, a, grid, smem, s);
        case 8: return launch_tc_d<8>(plan, a, grid, smem, s);
        case 16: return launch_tc_d<16>(plan, a, grid, smem, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace qst
