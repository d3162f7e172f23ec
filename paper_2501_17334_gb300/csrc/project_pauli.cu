// Structured form of the projector contraction for the Pauli POVMs (Sec. II, p_kl = Tr Lambda_kl
// rho, with Lambda_kl the Kronecker product over qubits of single-qubit eigenprojectors
// (1 +- P_q) / 2, P_q in {X, Y, Z}; Sec. IV uses all 3^Q settings), fused with the likelihood
// (Eq. likelihood) in the deviance form of the FP32 form.
//
// Because each projector is a product over qubits, the probabilities follow from rho by a tree
// over the qubits instead of a dense contraction.  Fixing the outcome of the most significant
// remaining qubit of a Hermitian block M = [[A, B], [B^dag, C]] (A: that qubit's bit 0 in row
// and column) leaves, on the other qubits, the Hermitian block Tr_q((Pi ⊗ 1) M):
//     X+-: (A + C +- (B + B^dag)) / 2,   Y+-: (A + C +- i (B - B^dag)) / 2,   Z+: A,   Z-: C.
// After Q such splits the 6^Q scalars are q_kl = Tr(Lambda_kl rho) of every setting and outcome.
// In the packed layout (Re rho_ij on and above the diagonal, Im rho_ij below it) a block's packed
// form is the same sub-block of its parent's packed form, and each entry of a child is a few
// real adds of parent entries (Re B_uv = TR_uv, Im B_uv = -BL_vu):
//     u <= v:  Re (B + B^dag)_uv = TR_uv + TR_vu,   Re i(B - B^dag)_uv = BL_uv + BL_vu
//     u >  v:  Im (B + B^dag)_uv = BL_uv - BL_vu,   Im i(B - B^dag)_uv = TR_uv - TR_vu
// with TR = the top-right and BL = the bottom-left quarter of the parent's packed form.  The tree
// costs about 3.5 * 6^Q adds per chain against the 2 * 24^Q FLOPs of the dense contraction;
// every add is one FP32 rounding and each value passes through Q of them.
//
// Work split: a chain's levels t = 0 .. Q-2 (6^t blocks of 2^(Q-t) x 2^(Q-t) packed floats, block
// index o = sum over split qubits of (2 s + b) 6^(...), the first split most significant) live
// in two shared-memory buffers (even levels in one, odd in the other; rows padded to n + 1 from
// n = 8 on, 4 x 4 blocks 20 floats apart).  A split task takes an entry pair (u, v), (v, u) of
// one parent (8 loads, 12 stores) or a diagonal entry.  The last two splits run in registers: a
// thread takes a 4 x 4 block of level Q-2 and forms its 36 outputs (tree indices 36 p .. 36 p +
// 35) and their deviance terms; a chain has one thread per block up to five qubits and 648
// threads with two blocks each at six.
// The deviance terms run on packed FP32 pairs (the outputs X+-, Y+-, Z+- of one split), with
// weights per pair: x = q w + a (w = P_k / count, halved for the X and Y pairs whose factor 1/2
// is left out of q, and w = 0, a = 1 for an outcome without counts, whose term is then 0); they
// are stored pair-major ([18][6^(Q-2)]) so that the threads of a warp read them coalesced.
//
// Every setting is renormalised by its own sum, log L = C0 + sum_k [sum_l c_kl log(q_kl / f_kl)
// - P_k log S_k], S_k = sum_l q_kl (the caller adds C0 - N log t, so the kernel adds
// -P_k log(S_k / t)).  For a complete POVM S_k = Tr rho = t in real arithmetic, so this is the
// likelihood of Eq. likelihood; in FP32 it cancels the part of each q's rounding error that is
// proportional to q, which near the posterior (c_kl ~ P_k p_kl) is most of its effect on log L.
// S_k - t is formed exactly: each q is split at 2^-20 (2^-19 for the doubled X, Y outputs) by
// adding and removing a constant, the high parts add without rounding and the low parts are
// tiny.  A thread sums the outcomes of the last two qubits for its 9 settings of them; the
// 2^(Q-2) threads of one setting prefix are combined in shared memory.
#include "qst_internal.cuh"
#include "f32x2.cuh"

namespace qst {
namespace {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int row_stride(int n) { return n >= 8 ? n + 1 : n; }   // of an n x n block
// floats per stored n x n block: the 4 x 4 blocks that one thread reads as four float4 rows sit
// 20 floats apart, so the 8 threads of a quarter warp cover all 32 banks
__host__ __device__ constexpr int block_floats(int n) { return n == 4 ? 20 : n * row_stride(n); }

template <int Q>
struct PauliShape {
    static constexpr int D = 1 << Q, d = D * D;
    // floats of level t: 6^t blocks of n x n, n = 2^(Q-t), rows padded to n + 1 from n = 8 on so
    // that the transposed reads of a split hit distinct banks
    static constexpr int level(int t) { return ipow(6, t) * block_floats(1 << (Q - t)); }
    static constexpr int max_level(int parity) {   // over the stored levels t <= Q - 2 of that parity
        int m = 0;
        for (int t = parity; t <= Q - 2; t += 2) m = cmax(m, level(t));
        return m;
    }
    static constexpr int NB = Q >= 2 ? ipow(6, Q - 2) : 1;   // 4 x 4 blocks of level Q - 2 per chain
    static constexpr int TPC = NB > 648 ? 648 : NB;          // threads per chain (each takes NB / TPC blocks)
    static constexpr int CPB = Q <= 2 ? 128 : (Q == 3 ? 48 : (Q == 4 ? 8 : 1));   // chains per CTA
    static constexpr int threads = TPC * CPB;                // 128, 128, 288, 288, 216, 648
    static constexpr int min_ctas = Q <= 2 ? 8 : (Q <= 4 ? 4 : (Q == 5 ? 5 : 1));   // per SM (a register cap)
    static constexpr int NS = Q == 1 ? 3 : 9;                // settings of the last one or two qubits
    // the setting sums (NS x NB (hi, lo) pairs per chain) take the odd-level buffer when the last
    // stored level is even (Q = 4, 6): it is dead by then
    static constexpr bool alias_spart = Q >= 4 && (Q % 2 == 0);
    // (hi, lo) pairs per setting slot of the sums: NB + 1, so that the 9 slots a warp's
    // consecutive settings read fall in different banks
    static constexpr int slot_stride = NB + 1;
    static constexpr int bufA = Q == 1 ? 4 : max_level(0);   // even levels (0: the packed rho)
    static constexpr int bufB = cmax(Q >= 3 ? max_level(1) : 0, alias_spart ? 2 * NS * slot_stride : 0);   // odd levels
    static constexpr int floats = (bufA + bufB + 3) / 4 * 4; // per chain
    static_assert(bufA % 4 == 0, "the odd levels' 4 x 4 blocks are read as float4 rows");
    static_assert(NB % TPC == 0, "whole blocks per thread");
};

struct PauliArgs {
    const float *A;          // [rows][d_pad] packed rho
    const float4 *wq;        // [18][6^(Q-2)] (w, w, a, a) of output pair 2 j, 2 j + 1 of block p at [j][p]
    const float2 *wc;        // [18][6^(Q-2)] their counts
    const int32_t *perm;     // [6^Q] tree order -> setting-major projector index
    const float *ptot;       // [3^Q] shots P_k of setting k
    double *out;             // [rows] the deviance sum (one column group)
    float *p_out;            // [rows][KD] (P_OUT only): p = q / t
    const double *trace;     // [rows] exact trace of the stored rho (P_OUT only)
    int64_t rows;
    int d_pad, KD;
    int poisson;             // 1: each setting adds -mu_k (S_k / t - 1) (Poisson; S_k / t - 1 is a few ulps
                             // here, the Pauli settings being complete) instead of -P_k log(S_k / t)
};

// The six children of one split at an entry: s = A + C, x = B + B^dag, y = i(B - B^dag) there.
__device__ __forceinline__ void six(float s, float x, float y, float a, float c, float o[6]) {
    o[0] = 0.5f * (s + x);
    o[1] = 0.5f * (s - x);
    o[2] = 0.5f * (s + y);
    o[3] = 0.5f * (s - y);
    o[4] = a;
    o[5] = c;
}

// One split of a level in shared memory: every parent (n x n) of `in` into its six children
// (h x h, h = n / 2) in `out`; tasks are the entry pairs u < v and the diagonal entries of the
// children, folded so that task r of h (h + 1) / 2 maps to row i = r / (h + 1) of the upper
// triangle and its complement row h - 1 - i.
template <int N>
__device__ __forceinline__ void split_level(const float *in, float *out, int parents, int lt, int tpc) {
    constexpr int h = N / 2, tasks = h * (h + 1) / 2;
    constexpr int PS = row_stride(N), CS = row_stride(h), hh = block_floats(h);   // row strides, child block size
    for (int idx = lt; idx < parents * tasks; idx += tpc) {
        const int p = idx / tasks, r = idx - p * tasks;
        const int i = r / (h + 1), j = r - i * (h + 1);
        const int u = (j < h - i) ? i : h - 1 - i;
        const int v = (j < h - i) ? i + j : h - 1 - i + (j - (h - i));
        const float *M = in + p * block_floats(N);
        float *O = out + 6 * p * hh;
        const float tl_uv = M[u * PS + v], br_uv = M[(h + u) * PS + h + v];
        const float tr_uv = M[u * PS + h + v], bl_uv = M[(h + u) * PS + v];
        float o[6];
        if (u == v) {
            six(tl_uv + br_uv, 2.0f * tr_uv, 2.0f * bl_uv, tl_uv, br_uv, o);
#pragma unroll
            for (int c = 0; c < 6; ++c) O[c * hh + u * CS + v] = o[c];
        } else {
            const float tl_vu = M[v * PS + u], br_vu = M[(h + v) * PS + h + u];
            const float tr_vu = M[v * PS + h + u], bl_vu = M[(h + v) * PS + u];
            six(tl_uv + br_uv, tr_uv + tr_vu, bl_uv + bl_vu, tl_uv, br_uv, o);          // (u, v): real parts
#pragma unroll
            for (int c = 0; c < 6; ++c) O[c * hh + u * CS + v] = o[c];
            six(tl_vu + br_vu, bl_vu - bl_uv, tr_vu - tr_uv, tl_vu, br_vu, o);          // (v, u): imaginary parts
#pragma unroll
            for (int c = 0; c < 6; ++c) O[c * hh + v * CS + u] = o[c];
        }
    }
}

// The last split of one 2 x 2 block [[e00, Re b], [Im b*, e11]] and the deviance terms of its
// six outputs, pairs j0 .. j0 + 2 of this thread's weights: (S +- 2 Re b), (S +- 2 Im b*) are
// 2 q of X+- and Y+- (the 1/2 sits in their weights), (e00, e11) are q of Z+-.
template <bool P_OUT>
__device__ __forceinline__ void last_split(float e00, float e01, float e10, float e11, const PauliArgs &a, int j0,
                                           int stride, int blk, float2 &dev, float2 &comp, int &xmin,
                                           float (&sh)[3], float (&sl)[3], float *p_row, int o0, float inv_t) {
    float4 wq[3];   // the three pairs' weights, requested before the arithmetic that needs them
    float2 wc[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        wq[j] = a.wq[(j0 + j) * stride + blk];
        wc[j] = a.wc[(j0 + j) * stride + blk];
    }
    const float S = e00 + e11;
    const float2 q2[3] = {fma2(splat2(e01), make_float2(2.0f, -2.0f), splat2(S)),
                          fma2(splat2(e10), make_float2(2.0f, -2.0f), splat2(S)), make_float2(e00, e11)};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float4 w = wq[j];
        const float2 cnt = wc[j];
        const float2 x = fma2(q2[j], make_float2(w.x, w.y), make_float2(w.z, w.w));
        xmin = min(xmin, min(__float_as_int(x.x), __float_as_int(x.y)));
        kahan_fma2(dev, comp, cnt, log_poly2(x));   // compensated: far from the posterior the terms are O(c)
        // the setting sum of this pair's q (2 q for X, Y): high parts on the grid, exactly
        const float2 C = splat2(j < 2 ? 24.0f : 12.0f);
        const float2 hq = sub2(add2(q2[j], C), C), lq = sub2(q2[j], hq);
        sh[j] += hq.x + hq.y;
        sl[j] += lq.x + lq.y;
        if constexpr (P_OUT) {
            if (p_row) {
                const float h = j < 2 ? 0.5f : 1.0f;
                p_row[a.perm[o0 + 2 * j]] = h * q2[j].x * inv_t;
                p_row[a.perm[o0 + 2 * j + 1]] = h * q2[j].y * inv_t;
            }
        }
    }
}

template <int Q, bool P_OUT, bool POISSON>
__global__ void __launch_bounds__(PauliShape<Q>::threads, PauliShape<Q>::min_ctas) project_pauli_kernel(PauliArgs a) {
    using S = PauliShape<Q>;
    constexpr int D = S::D, d = S::d, TPC = S::TPC, CPB = S::CPB, NB = S::NB;
    constexpr int NS = S::NS;
    extern __shared__ __align__(16) float smem[];
    __shared__ float part[S::threads], part_lo[S::threads];
    __shared__ float4 tinfo[CPB];                                   // (t_hi, t_lo, 1 / t_hi) per chain
    __shared__ float2 spart_s[(Q >= 3 && !S::alias_spart) ? CPB * NS * S::slot_stride : 1];   // setting sums per block
    const int g = threadIdx.x / TPC, lt = threadIdx.x - g * TPC;
    const int64_t c = (int64_t)blockIdx.x * CPB + g;
    const bool active = c < a.rows;
    float *bufA = smem + g * S::floats;
    float *bufB = bufA + S::bufA;
    // setting sums of chain g's blocks: [NS][NB + 1] (hi, lo)
    float2 *spart = S::alias_spart ? reinterpret_cast<float2 *>(bufB) : spart_s + g * NS * S::slot_stride;

    // t = t_hi + t_lo exactly (t is an FP64 sum of FP32 values, a few ulps from 1); the CTA's
    // chains in its first threads, so the few FP64 instructions fill their warps
    if (threadIdx.x < CPB) {
        const int64_t cc = (int64_t)blockIdx.x * CPB + threadIdx.x;
        const double t = cc < a.rows ? a.trace[cc] : 1.0;
        const float t_hi = (float)t;
        tinfo[threadIdx.x] = make_float4(t_hi, (float)(t - (double)t_hi), 1.0f / t_hi, 0.0f);
    }

    if (active)
        for (int e = 4 * lt; e < d; e += 4 * TPC) {
            const float4 r = *reinterpret_cast<const float4 *>(a.A + c * a.d_pad + e);
            float *row = bufA + (e / D) * row_stride(D) + e % D;   // (four entries of one row)
            row[0] = r.x;
            row[1] = r.y;
            row[2] = r.z;
            row[3] = r.w;
        }
    __syncthreads();

    // splits of the stored levels 0 .. Q-3
    if constexpr (Q >= 3) {
        split_level<D>(bufA, bufB, 1, lt, TPC);
        __syncthreads();
    }
    if constexpr (Q >= 4) {
        split_level<D / 2>(bufB, bufA, 6, lt, TPC);
        __syncthreads();
    }
    if constexpr (Q >= 5) {
        split_level<D / 4>(bufA, bufB, 36, lt, TPC);
        __syncthreads();
    }
    if constexpr (Q >= 6) {
        split_level<D / 8>(bufB, bufA, 216, lt, TPC);
        __syncthreads();
    }

    float2 dev = splat2(0.0f), comp = splat2(0.0f);   // deviance sum (dev - comp)
    int xmin = 0x7fffffff;   // smallest bit pattern of a log argument (sign included)
    float inv_t = 0.0f;
    float *p_row = nullptr;
    if constexpr (P_OUT) {
        inv_t = active ? (float)(1.0 / a.trace[c]) : 0.0f;
        p_row = active ? a.p_out + c * a.KD : nullptr;
    }
    const float4 ti = tinfo[g];
    // -P_k log(S_k / t) of a setting whose sums are (hi, lo) in units of `unit` q
    auto renorm = [&](float sh, float sl, float unit, int k) {
        const float rel = ((unit * sh - ti.x) + (unit * sl - ti.y)) * ti.z;
        // log1p(rel): |rel| is a few ulps, where three terms are exact to 2^-40
        if constexpr (POISSON) return -__ldg(a.ptot + k) * rel;   // (a compile-time choice)
        const float l1p = fabsf(rel) < 0x1p-10f ? rel * __fmaf_rn(rel, __fmaf_rn(rel, 0.33333334f, -0.5f), 1.0f)
                                                : log1pf(rel);
        return -__ldg(a.ptot + k) * l1p;
    };
    float extra = 0.0f;   // this thread's renormalisation terms
    float sh[3], sl[3];   // setting sums of the current child pair, per last-qubit setting j
#pragma unroll
    for (int j = 0; j < 3; ++j) sh[j] = sl[j] = 0.0f;
    if constexpr (Q == 1) {
        const float4 m = *reinterpret_cast<const float4 *>(bufA);   // [[a, Re b], [Im b*, e]]
        last_split<P_OUT>(m.x, m.y, m.z, m.w, a, 0, 1, 0, dev, comp, xmin, sh, sl, p_row, 0, inv_t);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            extra += renorm(sh[j], sl[j], j < 2 ? 0.5f : 1.0f, j);
    } else {
        // the last two splits of this thread's 4 x 4 blocks of level Q - 2 (blocks lt, lt + TPC, ..)
#pragma unroll 1
        for (int ib = 0; ib < NB / TPC; ++ib) {
            const int blk = lt + ib * TPC;
            const float *Mb = ((Q - 2) & 1 ? bufB : bufA) + block_floats(4) * blk;
            float M[16];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 v = *reinterpret_cast<const float4 *>(Mb + 4 * r);
                M[4 * r] = v.x;
                M[4 * r + 1] = v.y;
                M[4 * r + 2] = v.z;
                M[4 * r + 3] = v.w;
            }
            // first of the two: the 2 x 2 children at entries (0,0), (0,1), (1,0), (1,1)
            float e00[6], e01[6], e10[6], e11[6];
            six(M[0] + M[10], 2.0f * M[2], 2.0f * M[8], M[0], M[10], e00);
            six(M[1] + M[11], M[3] + M[6], M[9] + M[12], M[1], M[11], e01);
            six(M[4] + M[14], M[12] - M[9], M[6] - M[3], M[4], M[14], e10);
            six(M[5] + M[15], 2.0f * M[7], 2.0f * M[13], M[5], M[15], e11);
            // second: child c1 gives the outputs 36 blk + 6 c1 .. + 5, weight pairs 3 c1 .. 3 c1 + 2;
            // children 2 s and 2 s + 1 share the setting s of qubit Q - 2: after each such pair the
            // sums of settings (s, j) are complete for this block
#pragma unroll
            for (int c1 = 0; c1 < 6; ++c1) {
                last_split<P_OUT>(e00[c1], e01[c1], e10[c1], e11[c1], a, 3 * c1, NB, blk, dev, comp, xmin, sh, sl,
                                  p_row, 36 * blk + 6 * c1, inv_t);
                if (c1 & 1) {
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float2 v = make_float2(sh[j], sl[j]);
                        if constexpr (Q == 2) {
                            extra += renorm(v.x, v.y, j < 2 ? 0.5f : 1.0f, 3 * (c1 >> 1) + j);
                        } else {
                            spart[(3 * (c1 >> 1) + j) * S::slot_stride + blk] = v;
                        }
                        sh[j] = sl[j] = 0.0f;
                    }
                }
            }
        }
    }
    if constexpr (Q >= 3) {
        // the 2^(Q-2) threads of a setting prefix (same s_q, every b_q for q < Q - 2), in b order
        __syncthreads();
        constexpr int K3 = ipow(3, Q), NPRE = 1 << (Q - 2);   // settings; b-prefixes of a setting prefix
        for (int k = lt; k < K3; k += TPC) {
            const int slot = k % 9, pre = k / 9;   // (s_{Q-2}, s_{Q-1}) and the prefix's settings
            int base = 0;                           // thread of the prefix with every b_q = 0
#pragma unroll
            for (int q = 0; q < Q - 2; ++q) base += 2 * ((pre / ipow(3, Q - 3 - q)) % 3) * ipow(6, Q - 3 - q);
            const float2 *sp = spart + slot * S::slot_stride + base;
            float vh = 0.0f, vl = 0.0f;
#pragma unroll
            for (int b = 0; b < NPRE; ++b) {
                int off = 0;   // + sum_q b_q 6^(Q-3-q), a constant
#pragma unroll
                for (int q = 0; q < Q - 2; ++q) off += ((b >> (Q - 3 - q)) & 1) * ipow(6, Q - 3 - q);
                const float2 v = sp[off];
                vh += v.x;
                vl += v.y;
            }
            extra += renorm(vh, vl, slot % 3 < 2 ? 0.5f : 1.0f, k);
        }
    }
    // this thread's sum as an unevaluated pair (hi, lo): the two halves of the compensated sum
    // added exactly, the compensations and the small renormalisation terms in lo; a counted
    // outcome with q <= 0 (or below the normal range) makes log L = -inf
    float acc_hi, acc_lo;
    two_sum(dev.x, dev.y, acc_hi, acc_lo);
    acc_lo += extra - (comp.x + comp.y);
    if (xmin < 0x00800000) acc_hi = -INFINITY;

    // the chain's threads' pairs, added in thread order (two-sum of the high parts) by one thread
    // per chain; the CTA's chains sit in its first threads, so the FP64 result (scarce FP64
    // instructions, each costing its warp the same however many lanes are active) takes a few
    // warp instructions per CTA
    if constexpr (TPC == 1) {
        if (active) a.out[c] = (double)acc_hi + (double)acc_lo;
    } else {
        part[threadIdx.x] = acc_hi;
        part_lo[threadIdx.x] = acc_lo;
        __syncthreads();
        if (threadIdx.x < CPB) {
            const int64_t cc = (int64_t)blockIdx.x * CPB + threadIdx.x;
            float hi = 0.0f, lo = 0.0f;
            for (int t = 0; t < TPC; ++t) {
                float e;
                two_sum(hi, part[threadIdx.x * TPC + t], hi, e);
                lo += e + part_lo[threadIdx.x * TPC + t];
            }
            if (cc < a.rows) a.out[cc] = (double)hi + (double)lo;
        }
    }
}

template <int Q, bool P_OUT, bool POISSON>
cudaError_t launch_qpp(const PauliArgs &a, cudaStream_t s) {
    using S = PauliShape<Q>;
    const size_t smem = sizeof(float) * (size_t)S::floats * S::CPB;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(project_pauli_kernel<Q, P_OUT, POISSON>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t blocks = (a.rows + S::CPB - 1) / S::CPB;
    project_pauli_kernel<Q, P_OUT, POISSON><<<(unsigned)blocks, S::threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int Q, bool P_OUT>
cudaError_t launch_qp(const PauliArgs &a, cudaStream_t s) {
    return a.poisson ? launch_qpp<Q, P_OUT, true>(a, s) : launch_qpp<Q, P_OUT, false>(a, s);
}

template <int Q>
cudaError_t launch_q(const PauliArgs &a, cudaStream_t s) {
    return a.p_out ? launch_qp<Q, true>(a, s) : launch_qp<Q, false>(a, s);
}

}  // namespace

void pauli_tree_order(int Q, std::vector<int32_t> &perm) {
    const int D = 1 << Q, n = ipow(6, Q);
    perm.assign(n, 0);
    for (int o = 0; o < n; ++o) {
        int k = 0, l = 0, rest = o;
        for (int q = Q - 1; q >= 0; --q) {   // digit of qubit q: (o / 6^(Q-1-q)) % 6 = 2 s_q + b_q
            const int digit = rest % 6;
            rest /= 6;
            k += (digit / 2) * ipow(3, Q - 1 - q);
            l += (digit % 2) << (Q - 1 - q);
        }
        perm[o] = k * D + l;
    }
}

void pauli_weights(int Q, const std::vector<int32_t> &perm, const float *cnt, const float *invf,
                   std::vector<float4> &wq, std::vector<float2> &wc) {
    const int npb = Q >= 2 ? ipow(6, Q - 2) : 1;
    const int n = ipow(6, Q);
    wq.assign(n / 2, make_float4(0.f, 0.f, 1.f, 1.f));
    wc.assign(n / 2, make_float2(0.f, 0.f));
    for (int o = 0; o < n; ++o) {
        const int p = o / 36, k = o % 36;                 // block, output within the block
        const int j = k / 2, e = k % 2;                   // pair, element
        const int idx = j * npb + p;
        const float half = ((k % 6) < 4) ? 0.5f : 1.0f;   // X and Y outputs carry their 1/2 here
        const int m = perm[o];
        const bool counted = cnt[m] > 0.0f;
        float *q = reinterpret_cast<float *>(&wq[idx]);
        float *c = reinterpret_cast<float *>(&wc[idx]);
        q[e] = counted ? invf[m] * half : 0.0f;
        q[2 + e] = counted ? 0.0f : 1.0f;
        c[e] = cnt[m];
    }
}

cudaError_t launch_project_pauli(const ProblemView &p, const float *A, int64_t rows, double *out, float *p_out,
                                 cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    if (!p.pauli_wq || !p.pauli_wc || !p.pauli_perm) return cudaErrorInvalidValue;
    PauliArgs a;
    a.A = A;
    a.wq = p.pauli_wq;
    a.wc = p.pauli_wc;
    a.perm = p.pauli_perm;
    a.ptot = p.ptot;
    a.out = out;
    a.p_out = p_out;
    a.trace = p.trace_prop;
    a.rows = rows;
    a.d_pad = p.d_pad;
    a.KD = p.KD;
    a.poisson = p.poisson;
    switch (p.D) {
        case 2: return launch_q<1>(a, s);
        case 4: return launch_q<2>(a, s);
        case 8: return launch_q<3>(a, s);
        case 16: return launch_q<4>(a, s);
        case 32: return launch_q<5>(a, s);
        case 64: return launch_q<6>(a, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace qst
