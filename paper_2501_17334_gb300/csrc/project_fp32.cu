// Plain FP32 form of the projector contraction and log-likelihood (Sec. II,
// p_kl = Tr Lambda_kl rho; Eq. likelihood).
//
// p = A . P with A = packed vec_h(rho) rows [rows][d_pad] and P the packed projector
// matrix [d_pad][KD_pad].  A CTA owns 128 chains and sweeps a group of 128-column
// tiles; each thread keeps an 8 x 8 register tile.  The K sum runs in chunks of 32 terms:
// after each chunk the tile is added into a second-level sum (a thread-private array in
// shared memory) and restarted, so no FP32 chain is longer than 32 terms -- a 256-term chain
// rounds at the scale of its running sum 256 times, which at four qubits is most of the FP32
// form's log L error.  The epilogue evaluates the
// likelihood in deviance form, every setting k renormalised by its own sum S_k = sum_l q_kl,
//     log L = C0 - N log t + sum_k [ sum_{c_kl > 0} c_kl log(q_kl invf_kl) - P_k log(S_k / t) ],
// invf_kl = P_k / c_kl (q = vec_h(rho) . P, t the exact trace of the stored rho), which equals
// sum c log p exactly in real arithmetic (C0 = -sum c log invf; S_k = t for a complete POVM)
// and cancels the rounding the FP32 sums of a setting share.  S_k is summed exactly as a
// hi + lo pair over the four threads that hold the setting's 16 columns; each thread sums its
// deviance terms with a compensated (Kahan) sum carried as a pair into the FP64 combine of the
// 16 threads sharing a chain, and one FP64 partial per (column group, chain) is written.  The
// constant and trace terms are added by the accept kernel.
#include "qst_internal.cuh"
#include "f32x2.cuh"

namespace qst {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, kThreads = 256;
constexpr int kChunkSteps = 2;   // K steps of BK per chunk of the sum (32 terms)
// dynamic shared memory: the A and B stages, the column weights and the second-level sums
constexpr size_t kSmemBytes = sizeof(float) * (2 * BK * BM + 2 * BK * BN + 2 * BN + 64 * kThreads);

struct ProjectArgs {
    const float *A;      // [rows][d_pad]
    const float *P;      // [d_pad][KD_pad]
    const float *cnt;    // [KD_pad]
    const float *invf;   // [KD_pad]
    const float *ptot;   // [KD_pad / D] shots P_k of each setting
    double *out;         // [ngroups][rows]
    float *p_out;        // [rows][KD] or null: p = q / t
    const double *trace; // [rows] t, the exact trace of the stored rho (used only for p_out)
    int64_t rows;
    int d_pad, KD, KD_pad;
    int D;               // outcomes per setting (a setting's columns are consecutive)
    int tiles_per_group;
    int poisson;         // 1: each setting adds -mu_k (S_k / t - 1) (Poisson) instead of -P_k log(S_k / t)
};

// POISSON: the Poisson likelihood's setting term (a compile-time choice, so that the multinomial
// instantiation carries none of its code)
template <bool POISSON>
__global__ void __launch_bounds__(kThreads) project_fp32_kernel(ProjectArgs a) {
    extern __shared__ __align__(16) float dyn[];
    float (*As)[BK][BM] = reinterpret_cast<float (*)[BK][BM]>(dyn);
    float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(dyn + 2 * BK * BM);
    float *cnt_s = dyn + 2 * BK * BM + 2 * BK * BN, *invf_s = cnt_s + BN;
    float *tot = invf_s + BN;   // [64][kThreads]: element e of this thread's tile at e * kThreads + tid

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n_tiles_total = a.KD_pad / BN;
    const int t_begin = blockIdx.y * a.tiles_per_group;
    const int t_end = min(t_begin + a.tiles_per_group, n_tiles_total);

    // per row: the compensated deviance sum (sum - comp) and the small renormalisation terms
    float rowsum[8], rowcomp[8], rowsmall[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) rowsum[i] = rowcomp[i] = rowsmall[i] = 0.0f;
    float trace_hi[8], trace_lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
        const int64_t row = m0 + r;
        const double t = (row < a.rows) ? a.trace[row] : 1.0;
        trace_hi[i] = (float)t;
        trace_lo[i] = (float)(t - (double)trace_hi[i]);
    }

    const int k_steps = a.d_pad / BK;
    for (int nt = t_begin; nt < t_end; ++nt) {
        const int n0 = nt * BN;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.0f;

        // register staging for the next K slice
        float4 ra[2], rb[2];
        auto load_global = [&](int k0) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = tid + u * kThreads;   // 0..511
                const int r = idx / 4, q = idx % 4;
                const int64_t row = m0 + r;
                ra[u] = (row < a.rows) ? *reinterpret_cast<const float4 *>(a.A + row * a.d_pad + k0 + 4 * q)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                const int kk = idx / 32, cq = idx % 32;
                rb[u] = *reinterpret_cast<const float4 *>(a.P + (int64_t)(k0 + kk) * a.KD_pad + n0 + 4 * cq);
            }
        };
        auto store_shared = [&](int buf) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = tid + u * kThreads;
                const int r = idx / 4, q = idx % 4;
                As[buf][4 * q + 0][r] = ra[u].x;
                As[buf][4 * q + 1][r] = ra[u].y;
                As[buf][4 * q + 2][r] = ra[u].z;
                As[buf][4 * q + 3][r] = ra[u].w;
                const int kk = idx / 32, cq = idx % 32;
                *reinterpret_cast<float4 *>(&Bs[buf][kk][4 * cq]) = rb[u];
            }
        };

        if (tid < BN) {
            cnt_s[tid] = a.cnt[n0 + tid];
            invf_s[tid] = a.invf[n0 + tid];
        }
        load_global(0);
        store_shared(0);
        __syncthreads();
        for (int ks = 0; ks < k_steps; ++ks) {
            const int buf = ks & 1;
            if (ks + 1 < k_steps) load_global((ks + 1) * BK);
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = __fmaf_rn(av[i], bv[jj], acc[i][jj]);
            }
            if (ks + 1 < k_steps) {
                store_shared(buf ^ 1);
            }
            // end of a 32-term chunk (not the last one): fold the tile into the second-level sum
            if (ks % kChunkSteps == kChunkSteps - 1 && ks + 1 < k_steps) {
                const bool first = ks == kChunkSteps - 1;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        float *t = tot + (i * 8 + jj) * kThreads + tid;
                        *t = first ? acc[i][jj] : *t + acc[i][jj];
                        acc[i][jj] = 0.0f;
                    }
            }
            __syncthreads();
        }
        if (k_steps > kChunkSteps) {   // the last chunk joins the earlier ones
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) acc[i][jj] = tot[(i * 8 + jj) * kThreads + tid] + acc[i][jj];
        }

        // epilogue: deviance terms of this tile, and the renormalisation of its settings.  The
        // four columns jj = 4h .. 4h + 3 of this thread belong to one setting, whose other twelve
        // columns are held by the threads tx ^ 1, tx ^ 2, tx ^ 3 (16 columns per setting, D = 16;
        // for D < 16 a group of four columns holds whole settings, for D = 32 two groups of
        // threads form one setting)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
            const int64_t row = m0 + r;
            const float inv_tr = (a.p_out && row < a.rows) ? (float)(1.0 / a.trace[row]) : 0.0f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float sh = 0.0f, sl = 0.0f;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int jj = 4 * h + u;
                    const int col = (jj < 4) ? tx * 4 + jj : 64 + tx * 4 + (jj - 4);
                    const float pv = acc[i][jj];
                    const float cv = cnt_s[col];
                    if (cv > 0.0f) {   // Kahan: rowsum - rowcomp
                        const float y = __fmaf_rn(cv, deviance_log(pv * invf_s[col]), -rowcomp[i]);
                        const float tt = rowsum[i] + y;
                        rowcomp[i] = (tt - rowsum[i]) - y;
                        rowsum[i] = tt;
                    }
                    // S_k as an exact pair: every q in (-4, 4) split at 2^-20 (the hi parts add exactly)
                    const float hq = (pv + 12.0f) - 12.0f;
                    sh += hq;
                    sl += pv - hq;
                    if (a.p_out && row < a.rows && n0 + col < a.KD) a.p_out[row * a.KD + n0 + col] = pv * inv_tr;
                }
                // the setting's sum over the threads holding its columns (exact for the hi parts)
                const int col0 = (h == 0) ? tx * 4 : 64 + tx * 4;
                // threads per setting: D / 4 (1 .. 16, consecutive tx); at D = 2 a thread's four
                // columns hold two settings and the renormalisation is left out (the plain
                // deviance form alone is exact too)
                const int per = a.D / 4;
#pragma unroll
                for (int off = 1; off < 16; off <<= 1) {
                    if (off < per) {
                        sh += __shfl_xor_sync(0xffffffffu, sh, off);
                        sl += __shfl_xor_sync(0xffffffffu, sl, off);
                    }
                }
                if constexpr (POISSON) {
                    // Poisson: -mu_k (S_k / t - 1) per setting, its large part into the compensated
                    // sum; at D = 2 a thread's four columns are two whole settings
                    auto add_poisson = [&](float mu, float s_hi, float s_lo) {
                        float ph, pl;
                        poisson_setting(mu, s_hi, s_lo, trace_hi[i], trace_lo[i], ph, pl);
                        const float y = -ph - rowcomp[i];
                        const float tt = rowsum[i] + y;
                        rowcomp[i] = (tt - rowsum[i]) - y;
                        rowsum[i] = tt;
                        rowsmall[i] -= pl;
                    };
                    if (per >= 1) {
                        if ((tx & (per - 1)) == 0 && n0 + col0 < a.KD) add_poisson(a.ptot[(n0 + col0) / a.D], sh, sl);
                    } else {
#pragma unroll
                        for (int s2 = 0; s2 < 2; ++s2) {
                            if (n0 + col0 + 2 * s2 >= a.KD) continue;
                            float s_hi = 0.0f, s_lo = 0.0f;
#pragma unroll
                            for (int u = 2 * s2; u < 2 * s2 + 2; ++u) {
                                const float pv = acc[i][4 * h + u];
                                const float hq = (pv + 12.0f) - 12.0f;
                                s_hi += hq;
                                s_lo += pv - hq;
                            }
                            add_poisson(a.ptot[(n0 + col0 + 2 * s2) / 2], s_hi, s_lo);
                        }
                    }
                } else if (per >= 1 && (tx & (per - 1)) == 0 && n0 + col0 < a.KD) {   // (multinomial)
                    // one thread per setting adds -P_k log(S_k / t)
                    const float pk = a.ptot[(n0 + col0) / a.D];
                    const float rel = ((sh - trace_hi[i]) + (sl - trace_lo[i])) / trace_hi[i];
                    const float l1p = fabsf(rel) < 0x1p-10f
                                          ? rel * __fmaf_rn(rel, __fmaf_rn(rel, 0.33333334f, -0.5f), 1.0f)
                                          : log1pf(rel);
                    rowsmall[i] -= pk * l1p;
                }
            }
        }
        __syncthreads();   // cnt_s / invf_s reuse
    }

    // combine the 16 threads (tx) that share each row, in FP64
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        double v = ((double)rowsum[i] - (double)rowcomp[i]) + (double)rowsmall[i];
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
        const int64_t row = m0 + r;
        if (tx == 0 && row < a.rows) a.out[(int64_t)blockIdx.y * a.rows + row] = v;
    }
}

// ---- small problems (D <= 4, at most 32 settings, KD <= 128): one thread per (chain, setting) --
// The tiled kernel above is several thousand unrolled instructions; for a one- or two-qubit
// problem its few warps run them once per step from a cold instruction cache (about 40 us per
// launch for 64 one-qubit or 4096 two-qubit chains, most of it stalled on instruction fetch).  Here a thread
// forms its setting's D values q_kl = sum_i A_ri P_i,(kD+l) as one FMA chain over i (d <= 16
// terms), their deviance terms (compensated, as above), the setting's exact sum S_k and its
// renormalisation term, and the KP threads of a chain (KP >= K, a power of two, so that a chain's
// threads share a warp) add their partials in FP64 by shuffles: one partial per chain, the
// single column group this size has.  P (d x KD floats) is staged in shared memory.
template <int D, bool POISSON>
__global__ void __launch_bounds__(256) project_fp32_small_kernel(ProjectArgs a, int K, int KP) {
    constexpr int d = D * D;
    extern __shared__ __align__(16) float ps[];
    const int KD = a.KD;
    for (int e = threadIdx.x; e < d * KD; e += blockDim.x) ps[e] = a.P[(int64_t)(e / KD) * a.KD_pad + (e % KD)];
    __syncthreads();
    const int k = threadIdx.x % KP;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / KP) + threadIdx.x / KP;
    double v = 0.0;
    if (row < a.rows && k < K) {
        float ar[d];
#pragma unroll
        for (int i = 0; i < d; i += 4) {
            const float4 t4 = *reinterpret_cast<const float4 *>(a.A + row * a.d_pad + i);
            ar[i] = t4.x;
            ar[i + 1] = t4.y;
            ar[i + 2] = t4.z;
            ar[i + 3] = t4.w;
        }
        const double t = a.trace[row];
        const float t_hi = (float)t, t_lo = (float)(t - (double)t_hi);
        const float inv_tr = a.p_out ? (float)(1.0 / t) : 0.0f;
        float sum = 0.0f, comp = 0.0f, small = 0.0f, sh = 0.0f, sl = 0.0f;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const int col = k * D + l;
            float q = 0.0f;
#pragma unroll
            for (int i = 0; i < d; ++i) q = __fmaf_rn(ar[i], ps[i * KD + col], q);
            const float cv = a.cnt[col];
            if (cv > 0.0f) {   // Kahan: sum - comp
                const float y = __fmaf_rn(cv, deviance_log(q * a.invf[col]), -comp);
                const float tt = sum + y;
                comp = (tt - sum) - y;
                sum = tt;
            }
            const float hq = (q + 12.0f) - 12.0f;   // S_k as an exact pair, as above
            sh += hq;
            sl += q - hq;
            if (a.p_out) a.p_out[row * KD + col] = q * inv_tr;
        }
        if constexpr (POISSON) {   // -mu_k (S_k / t - 1)
            float ph, pl;
            poisson_setting(a.ptot[k], sh, sl, t_hi, t_lo, ph, pl);
            const float y = -ph - comp;
            const float tt = sum + y;
            comp = (tt - sum) - y;
            sum = tt;
            small -= pl;
        } else {   // -P_k log(S_k / t)
            const float rel = ((sh - t_hi) + (sl - t_lo)) / t_hi;
            const float l1p = fabsf(rel) < 0x1p-10f ? rel * __fmaf_rn(rel, __fmaf_rn(rel, 0.33333334f, -0.5f), 1.0f)
                                                    : log1pf(rel);
            small -= a.ptot[k] * l1p;
        }
        v = ((double)sum - (double)comp) + (double)small;
    }
    for (int off = 1; off < KP; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (k == 0 && row < a.rows) a.out[row] = v;
}

}  // namespace

int fp32_ngroups(const ProblemView &p, int64_t rows) {
    // enough CTAs to fill the machine: split the columns when there are few row tiles
    const int64_t mt = (rows + BM - 1) / BM;
    const int nt = p.KD_pad / BN;
    int g = 1;
    while (g < nt && mt * g < 2 * 152) g *= 2;
    return g > nt ? nt : g;
}

namespace {
template <bool POISSON>
cudaError_t launch_fp32(const ProjectArgs &a, dim3 grid, cudaStream_t s) {
    // more than 48 KB of dynamic shared memory: opted into once per device
    static unsigned long long attr_set = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && !((attr_set >> dev) & 1ull)) {
        e = cudaFuncSetAttribute(project_fp32_kernel<POISSON>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set |= 1ull << dev;
    }
    project_fp32_kernel<POISSON><<<grid, kThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_project_fp32(const ProblemView &p, const float *A, int64_t rows, double *out_part, float *p_out,
                                cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    if (p.KD_pad % BN != 0 || p.d_pad % BK != 0) return cudaErrorInvalidValue;
    ProjectArgs a;
    a.A = A;
    a.P = p.P32;
    a.cnt = p.cnt;
    a.invf = p.invf;
    a.ptot = p.ptot;
    a.D = p.D;
    a.out = out_part;
    a.p_out = p_out;
    a.trace = p.trace_prop;
    a.rows = rows;
    a.d_pad = p.d_pad;
    a.KD = p.KD;
    a.KD_pad = p.KD_pad;
    a.poisson = p.poisson;
    const int K = p.KD / p.D;
    if (p.D <= 4 && p.KD <= 128 && K <= 32 && p.ngroups == 1) {   // one column group: the small kernel
        int KP = 1;
        while (KP < K) KP <<= 1;
        const unsigned blocks = (unsigned)((rows + (256 / KP) - 1) / (256 / KP));
        const size_t smem = sizeof(float) * (size_t)p.D * p.D * p.KD;
        if (p.D == 2) {
            if (a.poisson) project_fp32_small_kernel<2, true><<<blocks, 256, smem, s>>>(a, K, KP);
            else project_fp32_small_kernel<2, false><<<blocks, 256, smem, s>>>(a, K, KP);
        } else {
            if (a.poisson) project_fp32_small_kernel<4, true><<<blocks, 256, smem, s>>>(a, K, KP);
            else project_fp32_small_kernel<4, false><<<blocks, 256, smem, s>>>(a, K, KP);
        }
        return cudaGetLastError();
    }
    const int nt = p.KD_pad / BN;
    const int groups = p.ngroups;
    a.tiles_per_group = (nt + groups - 1) / groups;
    dim3 grid((unsigned)((rows + BM - 1) / BM), (unsigned)groups);
    return a.poisson ? launch_fp32<true>(a, grid, s) : launch_fp32<false>(a, grid, s);
}

}  // namespace qst
