// Proposal and density-matrix assembly (Algorithm 2 l.3-4, Algorithm 1 l.2-6).
//
// One chain is handled by D consecutive lanes; lane j owns column j of the D x D
// blocks G and H (the latent layout is column-major, so a column is D contiguous
// floats of each of the four parts).  Per chain:
//   1. eta from Philox (tag 1, step j) and y' = sqrt(1 - beta^2) y + beta eta; y'
//      is written to the chain's other y buffer (the accept kernel flips to it);
//   2. modified Gram-Schmidt on the columns of H: lane k normalises column k and
//      publishes it, lanes j > k project it out.  MGS yields the unitary factor whose
//      R has a positive real diagonal, i.e. U = Q Lambda of Algorithm 1 l.5.  A second
//      pass over the result (PASSES = 2) re-orthogonalises it: Q1 = Q2 R2 with R2 upper
//      triangular with positive diagonal, so Q2 is still the same factor of H, and its
//      FP32 error drops from O(cond(H) 2^-24) loss of orthogonality to O(2^-24);
//   3. W = (U + I) G, lane j computing column j;
//   4. rho = W W^dag / Tr: lane a computes entries (a, a+t mod D) for t = 0..D/2
//      (the Hermitian half, balanced over lanes), packed as vec_h and scaled by the FP32
//      reciprocal of the trace.  The rounding of that scaling is not left in the
//      probabilities: the exact FP64 sum t of the *stored* FP32 diagonal (1 up to a few
//      ulps) is written too, and the likelihood uses p = (vec_h . P) / t, i.e. subtracts
//      N log t in FP64.  Then sum_l p_kl = 1 holds to the contraction's rounding, with no
//      coherent shift of every probability (which would cost N * 2^-24 in log L);
//   5. the packed row is stored as FP32 and, for the tensor-core contraction, as the
//      exact three-term bf16 split hi + mid + lo.
#include "qst_internal.cuh"

namespace qst {
namespace {

constexpr int kThreads = 256;

template <int D>
struct Shape {
    static constexpr int d = D * D;
    static constexpr int chains_per_block = kThreads / D;
    // per-chain shared memory: U then W (D x D complex) + packed rho (d floats) + pad
    static constexpr int smem_floats = 3 * D * D + 4;
};

template <int D>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int off = D / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

struct ProposeArgs {
    const float *x_eval;        // MODE_EVAL: [rows][nx] latent vectors
    float *y;                   // [2][R][nx]
    const uint8_t *cur;         // [R]
    const double *beta;         // [R]
    float *rho_out;             // [rows][d_pad] packed rho (FP32-normalised)
    __nv_bfloat16 *split_out;   // [rows][3][d_pad] or null
    double *trace_out;          // [rows] exact FP64 trace of the stored rho (1 up to rounding)
    float *rho_norm_out;        // MODE_EVAL, optional: [rows][d] copy of the packed rho
    int64_t rows;
    int64_t R;
    int64_t chain_offset;
    uint64_t seed;
    uint32_t step;
    int mode;
    int d_pad;
};

template <int D, int PASSES>
__global__ void __launch_bounds__(kThreads) propose_kernel(ProposeArgs a) {
    using S = Shape<D>;
    constexpr int d = S::d;
    constexpr int nx = 4 * d;
    extern __shared__ float smem[];

    const int j = threadIdx.x % D;       // owned column (and, in step 4, owned row)
    const int g = threadIdx.x / D;       // chain slot in the block
    const int64_t c = (int64_t)blockIdx.x * S::chains_per_block + g;
    const bool active = c < a.rows;
    float *sm = smem + g * S::smem_floats;
    float2 *mat = reinterpret_cast<float2 *>(sm);   // column-major complex D x D
    float *packed = sm + 2 * d;

    // ---- 1. latent proposal: the four D-long column slices this lane owns -----------------
    float yv[4][D];
    float coef_y = 1.0f, coef_eta = 0.0f;
    int cur = 0;
    if (active && a.mode == MODE_STEP) {
        cur = a.cur[c];
        const double b = a.beta[c];
        coef_y = (float)sqrt(1.0 - b * b);
        coef_eta = (float)b;
    } else if (a.mode == MODE_INIT) {
        coef_y = 0.0f;
        coef_eta = 1.0f;
    }
    const uint32_t chain_id = (uint32_t)(a.chain_offset + (active ? c : 0));
    const uint32_t tag = (a.mode == MODE_INIT) ? TAG_INIT : TAG_PROPOSAL;
    const uint32_t key_lo = (uint32_t)(a.seed & 0xffffffffu), key_hi = (uint32_t)(a.seed >> 32);
#pragma unroll
    for (int part = 0; part < 4; ++part) {
        const int base = part * d + j * D;   // element index of (row 0, column j)
        if (a.mode == MODE_EVAL) {
            const float *src = a.x_eval + (active ? c : 0) * nx + base;
#pragma unroll
            for (int i = 0; i < D; ++i) yv[part][i] = active ? src[i] : 0.0f;
            continue;
        }
        float y0[D];
        if (a.mode == MODE_STEP) {
            const float *src = a.y + ((int64_t)cur * a.R + (active ? c : 0)) * nx + base;
            if (D >= 4) {
#pragma unroll
                for (int i = 0; i < D; i += 4) {
                    const float4 v = active ? *reinterpret_cast<const float4 *>(src + i) : make_float4(0, 0, 0, 0);
                    y0[i] = v.x; y0[i + 1] = v.y; y0[i + 2] = v.z; y0[i + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i) y0[i] = active ? src[i] : 0.0f;
            }
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) y0[i] = 0.0f;
        }
        float eta[D];
        if (D >= 4) {
#pragma unroll
            for (int q = 0; q < D / 4; ++q) {
                const uint4 w = Philox::block(make_uint4((uint32_t)(base / 4 + q), a.step, chain_id, tag), key_lo, key_hi);
                Philox::gaussian_pair(w.x, w.y, eta[4 * q], eta[4 * q + 1]);
                Philox::gaussian_pair(w.z, w.w, eta[4 * q + 2], eta[4 * q + 3]);
            }
        } else {
            // D == 2: the column is half of block `part`; lane j takes uniform pair j
            const uint4 w = Philox::block(make_uint4((uint32_t)part, a.step, chain_id, tag), key_lo, key_hi);
            const uint32_t wu = (j == 0) ? w.x : w.z;
            const uint32_t wv = (j == 0) ? w.y : w.w;
            Philox::gaussian_pair(wu, wv, eta[0], eta[D - 1]);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) yv[part][i] = __fmaf_rn(coef_y, y0[i], coef_eta * eta[i]);
        if (active) {
            float *dst = a.y + ((int64_t)(1 - cur) * a.R + c) * nx + base;
            if (D >= 4) {
#pragma unroll
                for (int i = 0; i < D; i += 4)
                    *reinterpret_cast<float4 *>(dst + i) = make_float4(yv[part][i], yv[part][i + 1], yv[part][i + 2], yv[part][i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i) dst[i] = yv[part][i];
            }
        }
    }
    float(&gr)[D] = yv[0];
    float(&gi)[D] = yv[1];
    float(&hr)[D] = yv[2];
    float(&hi)[D] = yv[3];

    // ---- 2. modified Gram-Schmidt on the columns of H -> U (Algorithm 1 l.4-5) -----------
#pragma unroll 1
    for (int pass = 0; pass < PASSES; ++pass) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (j == k) {
            float nrm = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i) nrm = __fmaf_rn(hr[i], hr[i], __fmaf_rn(hi[i], hi[i], nrm));
            const float inv = 1.0f / sqrtf(nrm);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                hr[i] *= inv;
                hi[i] *= inv;
                mat[k * D + i] = make_float2(hr[i], hi[i]);
            }
        }
        __syncwarp();
        if (j > k) {
            float qr[D], qi[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const float2 q = mat[k * D + i];
                qr[i] = q.x;
                qi[i] = q.y;
            }
            float rr = 0.0f, ri = 0.0f;   // r = q^dag h
#pragma unroll
            for (int i = 0; i < D; ++i) {
                rr = __fmaf_rn(qr[i], hr[i], __fmaf_rn(qi[i], hi[i], rr));
                ri = __fmaf_rn(qr[i], hi[i], __fmaf_rn(-qi[i], hr[i], ri));
            }
#pragma unroll
            for (int i = 0; i < D; ++i) {
                hr[i] = __fmaf_rn(-rr, qr[i], __fmaf_rn(ri, qi[i], hr[i]));
                hi[i] = __fmaf_rn(-rr, qi[i], __fmaf_rn(-ri, qr[i], hi[i]));
            }
        }
    }
    __syncwarp();
    }

    // ---- 3. W = (U + I) G, column j: W[:,j] = G[:,j] + sum_k U[:,k] G[k,j] ------------------
    float wr[D], wi[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        wr[i] = gr[i];
        wi[i] = gi[i];
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float gkr = gr[k], gki = gi[k];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float2 u = mat[k * D + i];
            wr[i] = __fmaf_rn(u.x, gkr, __fmaf_rn(-u.y, gki, wr[i]));
            wi[i] = __fmaf_rn(u.x, gki, __fmaf_rn(u.y, gkr, wi[i]));
        }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < D; ++i) mat[j * D + i] = make_float2(wr[i], wi[i]);
    __syncwarp();

    // ---- 4. rho = W W^dag / Tr: lane a owns entries (a, a + t mod D), t = 0..D/2 ------------
    const int arow = j;
    float war[D], wai[D];
#pragma unroll
    for (int jj = 0; jj < D; ++jj) {
        const float2 w = mat[jj * D + arow];
        war[jj] = w.x;
        wai[jj] = w.y;
    }
    float diag = 0.0f;
#pragma unroll
    for (int jj = 0; jj < D; ++jj) diag = __fmaf_rn(war[jj], war[jj], __fmaf_rn(wai[jj], wai[jj], diag));
    const float inv_tr = (float)(1.0 / group_sum<D>((double)diag));
    const float diag_n = diag * inv_tr;
    const double trace = group_sum<D>((double)diag_n);   // exact sum of the stored diagonal
    packed[arow * D + arow] = diag_n;
#pragma unroll
    for (int t = 1; t <= D / 2; ++t) {
        const int b = (arow + t) & (D - 1);
        if (t == D / 2 && arow >= D / 2) continue;  // (a, a + D/2) is done by the lower lane
        float re = 0.0f, im = 0.0f;   // (W W^dag)_ab = sum_jj W[a,jj] conj(W[b,jj])
#pragma unroll
        for (int jj = 0; jj < D; ++jj) {
            const float2 wb = mat[jj * D + b];
            re = __fmaf_rn(war[jj], wb.x, __fmaf_rn(wai[jj], wb.y, re));
            im = __fmaf_rn(wai[jj], wb.x, __fmaf_rn(-war[jj], wb.y, im));
        }
        re *= inv_tr;
        im *= inv_tr;
        if (arow < b) {
            packed[arow * D + b] = re;
            packed[b * D + arow] = -im;
        } else {
            packed[arow * D + b] = im;
            packed[b * D + arow] = re;
        }
    }
    if (active && j == 0) a.trace_out[c] = trace;
    __syncwarp();

    // ---- 5. store packed rho (FP32) and its exact bf16 split ----------------------------------
    if (active) {
        float *dst = a.rho_out + c * a.d_pad;
        for (int e = 4 * j; e < d; e += 4 * D) {
            const float4 v = *reinterpret_cast<const float4 *>(packed + e);
            *reinterpret_cast<float4 *>(dst + e) = v;
            if (a.rho_norm_out) *reinterpret_cast<float4 *>(a.rho_norm_out + c * d + e) = v;
            if (a.split_out) {
                const float vv[4] = {v.x, v.y, v.z, v.w};
                __nv_bfloat16 hs[4], ms[4], ls[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    hs[u] = __float2bfloat16_rn(vv[u]);
                    const float r1 = vv[u] - __bfloat162float(hs[u]);
                    ms[u] = __float2bfloat16_rn(r1);
                    const float r2 = r1 - __bfloat162float(ms[u]);
                    ls[u] = __float2bfloat16_rn(r2);
                }
                __nv_bfloat16 *sp = a.split_out + c * 3 * (int64_t)a.d_pad + e;
                *reinterpret_cast<uint2 *>(sp) = *reinterpret_cast<const uint2 *>(hs);
                *reinterpret_cast<uint2 *>(sp + a.d_pad) = *reinterpret_cast<const uint2 *>(ms);
                *reinterpret_cast<uint2 *>(sp + 2 * a.d_pad) = *reinterpret_cast<const uint2 *>(ls);
            }
        }
    }
}

template <int D, int PASSES>
cudaError_t launch_propose_pd(const ProblemView &p, int mode, uint32_t step, const float *x_eval, int64_t rows,
                             bool want_split, float *rho_norm_out, cudaStream_t s) {
    using S = Shape<D>;
    ProposeArgs a;
    a.x_eval = x_eval;
    a.y = p.y;
    a.cur = p.cur;
    a.beta = p.beta;
    a.rho_out = p.rho_prop;
    a.split_out = want_split ? p.rho_split : nullptr;
    a.trace_out = p.trace_prop;
    a.rho_norm_out = (mode == MODE_EVAL) ? rho_norm_out : nullptr;
    a.rows = rows;
    a.R = p.R;
    a.chain_offset = p.chain_offset;
    a.seed = p.seed;
    a.step = step;
    a.mode = mode;
    a.d_pad = p.d_pad;
    const size_t smem = sizeof(float) * S::smem_floats * S::chains_per_block;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(propose_kernel<D, PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t blocks = (rows + S::chains_per_block - 1) / S::chains_per_block;
    if (blocks == 0) return cudaSuccess;
    propose_kernel<D, PASSES><<<(unsigned)blocks, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_propose_d(const ProblemView &p, int mode, uint32_t step, const float *x_eval, int64_t rows,
                             bool want_split, float *rho_norm_out, cudaStream_t s) {
    if (p.qr_passes == 1) return launch_propose_pd<D, 1>(p, mode, step, x_eval, rows, want_split, rho_norm_out, s);
    return launch_propose_pd<D, 2>(p, mode, step, x_eval, rows, want_split, rho_norm_out, s);
}

}  // namespace

cudaError_t launch_propose(const ProblemView &p, int mode, uint32_t step, const float *x_eval, int64_t n_eval,
                           bool want_split, float *rho_norm_out, uint32_t *status, cudaStream_t s) {
    (void)status;
    const int64_t rows = (mode == MODE_EVAL) ? n_eval : p.R;
    switch (p.D) {
        case 2: return launch_propose_d<2>(p, mode, step, x_eval, rows, want_split, rho_norm_out, s);
        case 4: return launch_propose_d<4>(p, mode, step, x_eval, rows, want_split, rho_norm_out, s);
        case 8: return launch_propose_d<8>(p, mode, step, x_eval, rows, want_split, rho_norm_out, s);
        case 16: return launch_propose_d<16>(p, mode, step, x_eval, rows, want_split, rho_norm_out, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qst
