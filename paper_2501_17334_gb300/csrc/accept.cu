// Accept / reject, step-size adaptation, thinning and pooling (Algorithm 2,
// Eq. BME2), the diagnostics reductions (Eq. ACFrho, Eq. IACT) and small test hooks.
#include "qst_internal.cuh"

namespace qst {
namespace {

constexpr int kChainsPerCta = 128;   // the most chains one accept CTA takes (ProblemView::accept_cpc)
constexpr int kThreads = 256;

struct AcceptArgs {
    ProblemView p;
    SamplerParams sp;
    int mode;          // MODE_INIT or MODE_STEP
    uint32_t step;     // j
    int kept;          // j is a kept step (j % T == 0 and j > burn_in)
    int64_t kept_idx;  // index of this kept state (0-based) in the trajectories
    const StepState *step_dev;   // when not null: step, kept and kept_idx come from here
};

// One CTA owns chains [C b, C b + C) and pool slot b, C = p.accept_cpc <= 128.
__global__ void __launch_bounds__(kThreads) accept_kernel(AcceptArgs a) {
    const ProblemView &p = a.p;
    if (a.step_dev) {   // (a is this thread's copy of the parameters)
        a.step = a.step_dev->step;
        a.kept = a.step_dev->kept;
        a.kept_idx = a.step_dev->kept_idx;
    }
    __shared__ uint8_t flag[kChainsPerCta];
    __shared__ float inv_tr[kChainsPerCta];
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * p.accept_cpc;
    const int nc = (int)min((int64_t)p.accept_cpc, p.R - c0);

    // ---- phase 1: one thread per chain -------------------------------------------------
    if (tid < kChainsPerCta) {
        uint8_t acc = 0;
        float itr = 0.0f;
        if (tid < nc) {
            const int64_t c = c0 + tid;
            // log L(y') = C0 + sum_{c>0} c log(q invf) - N log t: q = vec_h(rho) . P for the
            // stored FP32 rho, t its exact trace, p = q / t
            const double tr = p.trace_prop[c];
            itr = 1.0f / (float)tr;
            // log t: t is the exact trace of an already normalised rho, so |t - 1| is a few ulps;
            // three terms of log1p(t - 1) then leave less than (t - 1)^4 / 4, far below FP64
            // rounding (FP64 log would cost ~30 of the scarce FP64 FMAs; it is kept for
            // |t - 1| >= 2^-10)
            const double dl = tr - 1.0;
            double logl_prop = p.C0 - p.Ntot * (fabs(dl) < 0x1p-10 ? dl * (1.0 - dl * (0.5 - dl * (1.0 / 3.0))) : log(tr));
            for (int g = 0; g < p.ngroups; ++g) logl_prop += p.logl_part[(int64_t)g * p.R + c];
            if (a.mode == MODE_INIT) {
                acc = 1;
                p.logl_cur[c] = logl_prop;
                p.cur[c] = 1;   // the initial proposal always lands in slot 1
            } else {
                // accept test: alpha ~ U(0,1), accept iff log alpha < log L(y') - log L(y)
                const uint32_t chain_id = (uint32_t)(p.chain_offset + c);
                const uint4 w = Philox::block(make_uint4(0u, a.step, chain_id, TAG_ALPHA),
                                              (uint32_t)(p.seed & 0xffffffffu), (uint32_t)(p.seed >> 32));
                const float alpha = ((float)(w.x >> 9) + 0.5f) * 0x1p-23f;
                // log alpha in FP32 (alpha is exact in FP32; error <= 2e-6, far inside the
                // near-tie band); the log-ratio it is compared with stays FP64
                const double log_alpha = (double)logf(alpha);
                const double logl_cur = p.logl_cur[c];
                acc = (log_alpha < logl_prop - logl_cur) ? 1 : 0;
                int32_t win = p.acc_win[c];
                if (acc) {
                    p.logl_cur[c] = logl_prop;
                    p.cur[c] ^= 1;
                    win += 1;
                    p.acc_total[c] += 1;
                }
                if (p.trace_steps > 0 && a.step >= 1 && a.step <= (uint32_t)p.trace_steps) {
                    const int64_t t = (int64_t)(a.step - 1) * p.R + c;
                    p.trace_acc[t] = acc;
                    p.trace_logl[t] = logl_prop;
                }
                // adaptation: every M_A steps rescale beta by the window's acceptance rate
                if (a.sp.adapt_interval > 0 && a.step % (uint32_t)a.sp.adapt_interval == 0) {
                    const double rate = (double)win / (double)a.sp.adapt_interval;
                    double beta = p.beta[c];
                    if (rate > a.sp.acc_hi) beta = a.sp.adapt_factor * beta;
                    if (rate < a.sp.acc_lo) beta = beta / a.sp.adapt_factor;
                    if (beta > a.sp.beta_max) beta = a.sp.beta_max;
                    p.beta[c] = beta;
                    p.coef[c] = make_float2((float)sqrt(1.0 - beta * beta), (float)beta);
                    win = 0;
                }
                p.acc_win[c] = win;
            }
        }
        flag[tid] = acc;
        inv_tr[tid] = itr;
    }
    __syncthreads();

    // ---- phase 2: rho write-back, pooling of the current state, trajectories ------------
    // Thread t moves float4 number (t mod V) of a chain's packed rho (V = d/4 per chain) for
    // the chains t/V, t/V + P, ... (P = 256/V chains in flight per pass, four passes
    // unrolled so that several independent loads are outstanding).  Pool sums: per-thread
    // float4 partials, then a shared-memory reduction over the P chain lanes.
    const int d = p.d;
    const int V = d / 4;
    const int P = kThreads / V < 1 ? 1 : kThreads / V;
    const bool pool_now = (a.mode == MODE_STEP) && a.kept;
    const int vi = tid % V, lane_c = tid / V;
    __shared__ float4 red4[kThreads];
    for (int v0 = 0; v0 < V; v0 += kThreads) {          // d > 1024 only: several vector columns per thread
        const int vv = v0 + (V < kThreads ? vi : tid);
        const bool vthread = (V < kThreads) ? (lane_c < P) : (vv < V);
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        if (vthread) {
            // chains k0, k0 + st, ...: four loads in flight per batch, one per chain (the new
            // current state: rho' if accepted, else the stored rho, read only when pooling)
            const int k0 = (V < kThreads ? lane_c : 0), st = (V < kThreads ? P : 1);
            constexpr int B = 4;
            for (int kb = k0; kb < nc; kb += B * st) {
                float4 q[B];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const int k = kb + u * st;
                    q[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k < nc && (flag[k] || pool_now)) {
                        const int64_t c = c0 + k;
                        const float *row = flag[k] ? p.rho_prop : p.rho_cur;
                        q[u] = reinterpret_cast<const float4 *>(row + c * p.d_pad)[vv];
                    }
                }
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const int k = kb + u * st;
                    if (k >= nc) break;
                    const int64_t c = c0 + k;
                    float4 val = q[u];
                    if (flag[k]) {
                        const float s_ = inv_tr[k];
                        val = make_float4(val.x * s_, val.y * s_, val.z * s_, val.w * s_);
                        reinterpret_cast<float4 *>(p.rho_cur + c * p.d_pad)[vv] = val;
                    }
                    if (pool_now) {
                        sum.x += val.x;
                        sum.y += val.y;
                        sum.z += val.z;
                        sum.w += val.w;
                        if (c < p.n_diag && a.kept_idx < p.traj_cap)
                            reinterpret_cast<float4 *>(p.traj + ((int64_t)c * p.traj_cap + a.kept_idx) * d)[vv] = val;
                    }
                }
            }
        }
        if (pool_now) {
            red4[tid] = sum;
            __syncthreads();
            if (V < kThreads) {
                if (tid < V) {
                    float4 tot = red4[tid];
                    for (int q = 1; q < P; ++q) {
                        const float4 o = red4[q * V + tid];
                        tot.x += o.x;
                        tot.y += o.y;
                        tot.z += o.z;
                        tot.w += o.w;
                    }
                    double *slot = p.pool + (int64_t)blockIdx.x * d + 4 * tid;
                    slot[0] += (double)tot.x;
                    slot[1] += (double)tot.y;
                    slot[2] += (double)tot.z;
                    slot[3] += (double)tot.w;
                }
            } else if (vthread) {
                double *slot = p.pool + (int64_t)blockIdx.x * d + 4 * vv;
                slot[0] += (double)sum.x;
                slot[1] += (double)sum.y;
                slot[2] += (double)sum.z;
                slot[3] += (double)sum.w;
            }
            __syncthreads();
        }
        if (V < kThreads) break;
    }
}

// Sums the pool slots -> out[d] (deterministic): a CTA owns 32 consecutive entries; its warp w
// adds slots [w n/32, (w + 1) n/32) in slot order, and the 32 partial sums are added in warp order.
constexpr int kReduceWarps = 32;
__global__ void __launch_bounds__(32 * kReduceWarps) pool_reduce_kernel(const double *pool, int n_slots, int d,
                                                                          double *out) {
    __shared__ double part[kReduceWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    const int per = (n_slots + kReduceWarps - 1) / kReduceWarps;
    const int b0 = w * per, b1 = min(n_slots, b0 + per);
    double s = 0.0;
    if (e < d)
        for (int b = b0; b < b1; ++b) s += pool[(int64_t)b * d + e];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < d) {
        double t = 0.0;
        for (int k = 0; k < kReduceWarps; ++k) t += part[k][lane];
        out[e] = t;
    }
}

// Eq. ACFrho for one diagnostic chain per CTA: c~[l] = sum_{n < N - lmax} sum_e w_e
// (x_n,e - m_e)(x_{n+l},e - m_e) with w_e = 1 on the diagonal and 2 off it (each packed
// off-diagonal entry stands for the (i,j) and (j,i) terms of Eq. ACFa).  Products in
// FP32 summed over chunks of 32 samples, chunks accumulated in FP64.
__global__ void acf_kernel(const float *traj, int traj_cap, int d, int D, int n_kept, int lmax, double *out) {
    extern __shared__ float sh[];  // mean[d]
    __shared__ double red[kThreads];
    const float *x = traj + (int64_t)blockIdx.x * traj_cap * d;
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        double s = 0.0;
        for (int n = 0; n < n_kept; ++n) s += x[(int64_t)n * d + e];
        sh[e] = (float)(s / n_kept);
    }
    __syncthreads();
    const int m = n_kept - lmax;
    for (int l = 0; l <= lmax; ++l) {
        double acc = 0.0;
        for (int e = threadIdx.x; e < d; e += blockDim.x) {
            const float mu = sh[e];
            const float w = ((e / D) == (e % D)) ? 1.0f : 2.0f;
            float chunk = 0.0f;
            for (int n = 0; n < m; ++n) {
                chunk = __fmaf_rn(x[(int64_t)n * d + e] - mu, x[(int64_t)(n + l) * d + e] - mu, chunk);
                if ((n & 31) == 31) {
                    acc += (double)(w * chunk);
                    chunk = 0.0f;
                }
            }
            acc += (double)(w * chunk);
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[(int64_t)blockIdx.x * (lmax + 1) + l] = red[0];
        __syncthreads();
    }
}

// log L = C0 - N log t + sum over column groups, for stateless evaluation.
__global__ void logl_combine_kernel(const double *part, const double *trace, int ngroups, int64_t rows, double C0,
                                    double Ntot, double *out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double v = C0 - Ntot * log(trace[r]);
    for (int g = 0; g < ngroups; ++g) v += part[(int64_t)g * rows + r];
    out[r] = v;
}

__global__ void philox_blocks_kernel(uint64_t seed, uint32_t step, uint32_t tag, uint32_t chain0, int64_t nchains,
                                     uint32_t block0, int32_t nblocks, uint32_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nchains * nblocks) return;
    const uint32_t c = chain0 + (uint32_t)(i / nblocks);
    const uint32_t b = block0 + (uint32_t)(i % nblocks);
    const uint4 w = Philox::block(make_uint4(b, step, c, tag), (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    reinterpret_cast<uint4 *>(out)[i] = w;
}

__global__ void inject_nan_kernel(float *y, const uint8_t *cur, int64_t R, int nx, int64_t chain) {
    const int b = cur[chain];
    for (int e = threadIdx.x; e < nx; e += blockDim.x) y[((int64_t)b * R + chain) * nx + e] = __int_as_float(0x7fc00000);
}

// Opens step j = step + 1 (one thread): whether j is kept and at which index.
__global__ void advance_step_kernel(StepState *st, int thin, int burn_in) {
    const uint32_t j = st->step + 1u;
    const int kept = (j % (uint32_t)thin == 0u) && ((int64_t)j > (int64_t)burn_in);
    st->step = j;
    st->kept = kept;
    st->kept_idx = st->kept_count;
    st->kept_count += kept;
}

}  // namespace

cudaError_t launch_advance_step(StepState *st, int thin, int burn_in, cudaStream_t s) {
    advance_step_kernel<<<1, 1, 0, s>>>(st, thin, burn_in);
    return cudaGetLastError();
}

cudaError_t launch_accept(const ProblemView &p, const SamplerParams &sp, int mode, const StepState *step_dev, uint32_t step,
                          bool kept, int64_t kept_idx, uint32_t *status, cudaStream_t s) {
    (void)status;
    AcceptArgs a;
    a.p = p;
    a.sp = sp;
    a.mode = mode;
    a.step = step;
    a.kept = kept ? 1 : 0;
    a.kept_idx = kept_idx;
    a.step_dev = step_dev;
    const int64_t blocks = (p.R + p.accept_cpc - 1) / p.accept_cpc;
    accept_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// Up to 256 packed floats per chain (D <= 16) a CTA takes 128 chains, which moves its 256
// threads' float4 lanes over several chains at once.  From D = 32 on, each chain alone fills
// the CTA's lanes and a CTA walks its chains in turn, so 128 chains per CTA leave most SMs
// idle (4096 six-qubit chains: 32 CTAs) and the copy latency-bound: halve the chains per CTA
// until the grid covers the SMs twice, down to 8 (more pool slots, each read and written
// once per kept step).
int accept_chains_per_cta(int64_t R, int d) {
    if (d < 4 * kThreads) return kChainsPerCta;
    static int num_sms = 0;
    if (num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms <= 0)
            num_sms = 148;
    }
    int c = kChainsPerCta;
    while (c > 8 && (R + c - 1) / c < 2 * (int64_t)num_sms) c /= 2;
    return c;
}

cudaError_t launch_pool_reduce(const ProblemView &p, double *out, cudaStream_t s) {
    pool_reduce_kernel<<<(p.d + 31) / 32, 32 * kReduceWarps, 0, s>>>(p.pool, p.n_slots, p.d, out);
    return cudaGetLastError();
}

cudaError_t launch_acf(const ProblemView &p, int n_kept, int lmax, double *acf_raw, cudaStream_t s) {
    if (p.n_diag <= 0 || n_kept <= lmax) return cudaSuccess;
    acf_kernel<<<p.n_diag, kThreads, sizeof(float) * p.d, s>>>(p.traj, p.traj_cap, p.d, p.D, n_kept, lmax, acf_raw);
    return cudaGetLastError();
}

cudaError_t launch_logl_combine(const ProblemView &p, int64_t rows, double *out, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    logl_combine_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(p.logl_part, p.trace_prop, p.ngroups, rows, p.C0,
                                                                         p.Ntot, out);
    return cudaGetLastError();
}

cudaError_t launch_philox_blocks(uint64_t seed, uint32_t step, uint32_t tag, uint32_t chain0, int64_t nchains,
                                 uint32_t block0, int32_t nblocks, uint32_t *out, cudaStream_t s) {
    const int64_t total = nchains * nblocks;
    if (total <= 0) return cudaSuccess;
    philox_blocks_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(seed, step, tag, chain0, nchains, block0,
                                                                          nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_inject_nan(const ProblemView &p, int64_t chain, cudaStream_t s) {
    inject_nan_kernel<<<1, 256, 0, s>>>(p.y, p.cur, p.R, p.nx, chain);
    return cudaGetLastError();
}

}  // namespace qst
