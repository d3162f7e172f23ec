// Proposal and density-matrix assembly (the proposal of Algorithm 2, Algorithm 1).
//
// One chain is handled by D consecutive lanes; lane j owns column j of the D x D
// blocks G and H (the latent layout is column-major, so a column is D contiguous
// floats of each of the four parts).  Per chain:
//   1. eta from Philox (tag 1, step j) and y' = sqrt(1 - beta^2) y + beta eta, one
//      Philox block (four entries) at a time; y' goes to the chain's other y buffer (the
//      accept kernel flips to it); lane j keeps H's column j in registers.  G's column is
//      read back from those same (own) global writes in step 3.
//   2. QR of H (Algorithm 1).  Modified Gram-Schmidt: at step k lane k publishes its
//      (unnormalised) column v_k, and every lane j > k loads it, forms |v_k|^2 and v_k^dag h_j
//      itself and removes the projection -- no lane works alone on a normalisation.  The
//      columns are normalised at the end.  MGS yields the unitary factor whose R has a
//      positive real diagonal, i.e. U = Q Lambda of Algorithm 1.  Its FP32 columns are
//      orthogonal only to O(cond(H) 2^-24); with PASSES = 2 they are re-orthogonalised once:
//      Q1 = Q2 R2 with R2 = chol(Q1^dag Q1) = I + F + O(E^2), E = Q1^dag Q1 - I,
//      F = strict upper part of E plus half its (real) diagonal, so Q2 = Q1 (I - F) is the
//      same QR factor of H to O(E^2) (E < 1e-4 after one pass for cond(H) < 1e4, so E^2
//      is below FP32 rounding).  Unlike a second Gram-Schmidt sweep this is two balanced
//      products: lane a forms entries (a, a + t) of E, then row a of Q1 (I - F).
//   3. W = (U + I) G, lane j computing column j;
//   4. rho = W W^dag / Tr: lane a computes entries (a, a+t mod D) for t = 0..D/2
//      (the Hermitian half, balanced over lanes), packed as vec_h and scaled by the FP32
//      reciprocal of the trace.  The rounding of that scaling is not left in the
//      probabilities: the exact sum t of the *stored* FP32 diagonal (1 up to a few ulps,
//      formed by a TwoSum reduction) is written too, and the likelihood uses
//      p = (vec_h . P) / t, i.e. subtracts N log t in FP64.  Then sum_l p_kl = 1 holds to
//      the contraction's rounding, with no coherent shift of every probability (which
//      would cost N * 2^-24 in log L);
//   5. the packed row is stored as FP32 and, for the tensor-core contraction, as the
//      exact three-term bf16 split hi + mid + lo.
#include "qst_internal.cuh"
#include "f32x2.cuh"

namespace qst {
namespace {

constexpr int kThreads = 128;
// the refinement of U (PASSES = 3): at most this many first-order passes, another one while the
// chain's largest |Y| entry exceeds kRefineTol (the residual of a pass is about |Y|^2)
constexpr int kRefinePasses = 3;
constexpr float kRefineTol = 0x1p-13f;

// The refinement keeps Q's and H's columns unpadded at D = 16 (16 floats each, so that five CTAs
// fit on an SM), where the 16 lanes of a chain reaching block b of their own columns would hit
// 8 of the 32 banks.  So block b (4 floats) of Q's column c is stored at b ^ ((c >> 1) & 3), and
// of H's column c at b ^ ((c >> 1) & 3) ^ 2: a chain's lanes then cover all 32 banks, and the Q
// and H columns of one index, which the refinement's products read side by side, never share
// banks.  Within a block the order is kept, so every value and every result is unchanged.
// (QC == D only for that layout; every other one is padded and unswizzled.)
template <int D, int QC>
__device__ __forceinline__ int qsw(int c) { return (QC == D && D == 16) ? ((c >> 1) & 3) : 0; }
template <int D, int QC>
__device__ __forceinline__ int hsw(int c) { return (QC == D && D == 16) ? (((c >> 1) & 3) ^ 2) : 0; }

// Shared memory per chain (floats), laid out so every access is free of bank conflicts:
//   area A: the real and imaginary planes of H's columns as they are orthogonalised (column
//           stride D + 4, so that 128-bit accesses of eight consecutive lanes' columns hit
//           different banks) -> W row-major (complex, rows padded to D + 2) once U is no
//           longer needed;
//   area B: F, dense complex column-major (only i <= j + 1 is written and read) -> packed
//           rho (row stride D + 1).
// The per-chain stride is an odd multiple of 16 floats, so the two chains of a warp that
// read the same offset in their own areas use opposite halves of the banks.
//   area R (PASSES = 3 only): the upper triangle of R from the Gram-Schmidt sweep, packed
//           (column c, row k <= c at c (c + 1) / 2 + k, complex), which the refinement's
//           triangular solve reads; area B then holds H's original columns during the
//           refinement's products.  At D = 16 the Q planes are unpadded there (area A stays at
//           W's 576 floats), which keeps five CTAs on an SM.

template <int D, int PASSES = 2, int THREADS = kThreads>
struct Shape {
    static constexpr int d = D * D;
    static constexpr int chains_per_block = THREADS / D;
    static constexpr int row_stride = D + 2;                    // float2 per row of W (padded)
    static constexpr int qcol = (PASSES == 3 && D == 16) ? D : D + 4;   // floats per column of a Q plane
    static constexpr int pk_stride = D + 1;                     // floats per row of the staged rho
    static constexpr int area_a = (2 * D * qcol > 2 * D * row_stride) ? 2 * D * qcol : 2 * D * row_stride;
    static constexpr int area_b = (2 * D * D > D * pk_stride) ? 2 * D * D : D * pk_stride;
    static constexpr int area_r = (PASSES == 3) ? D * (D + 1) : 0;
    static constexpr int raw = area_a + area_b + area_r;
    static constexpr int smem_floats = (raw + 31) / 32 * 32 + 16;
};

// Box-Muller with the fast hardware log, reciprocal square root and sine/cosine: the angle is
// reduced to 2 pi (v - 1/2) in (-pi, pi), where the intrinsics are accurate to ~2^-21
// absolute, and cos/sin(2 pi v) = -cos/-sin(2 pi (v - 1/2)).  v - 1/2 is exact.  The radius
// sqrt(t), t = -2 ln u >= 2^-23, is t rsqrt(t) (a few ulps).  The normals agree with the FP64
// Box-Muller of the same uniforms to about 1e-6 relative.
__device__ __forceinline__ void gaussian_pair_fast(uint32_t wu, uint32_t wv, float &z0, float &z1) {
    const float u = Philox::uniform(wu);
    const float v = Philox::uniform(wv);
    const float t = -2.0f * __logf(u);
    const float radius = t * rsqrtf(t);
    float s, c;
    __sincosf(6.283185307179586f * (v - 0.5f), &s, &c);
    z0 = -radius * c;
    z1 = -radius * s;
}

// a D-float column into / from registers, 128-bit at a time where D allows
template <int D>
__device__ __forceinline__ void load_column(const float *src, float (&v)[D], int s = 0) {
    if constexpr (D >= 4) {
#pragma unroll
        for (int i = 0; i < D; i += 4) {
            const float4 t = *reinterpret_cast<const float4 *>(src + 4 * ((i / 4) ^ s));
            v[i] = t.x;
            v[i + 1] = t.y;
            v[i + 2] = t.z;
            v[i + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) v[i] = src[i];
    }
}
template <int D>
__device__ __forceinline__ void store_column(float *dst, const float (&v)[D]) {
    if constexpr (D >= 4) {
#pragma unroll
        for (int i = 0; i < D; i += 4)
            *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) dst[i] = v[i];
    }
}

// a D-float column as D/2 pairs of consecutive entries (for the packed f32x2 arithmetic).  `s`:
// the column's 4-float blocks are stored in the order b ^ s (the swizzle of the unpadded
// 16-float columns of the refinement, kSwizzle below; 0 elsewhere)
template <int D>
__device__ __forceinline__ void load_column2(const float *src, float2 (&v)[D / 2], int s = 0) {
    if constexpr (D >= 4) {
#pragma unroll
        for (int p = 0; p < D / 2; p += 2) {
            const float4 t = *reinterpret_cast<const float4 *>(src + 4 * ((p / 2) ^ s));
            v[p] = make_float2(t.x, t.y);
            v[p + 1] = make_float2(t.z, t.w);
        }
    } else {
        v[0] = *reinterpret_cast<const float2 *>(src);
    }
}
template <int D>
__device__ __forceinline__ void store_column2(float *dst, const float2 (&v)[D / 2], int s = 0) {
    if constexpr (D >= 4) {
#pragma unroll
        for (int p = 0; p < D / 2; p += 2)
            *reinterpret_cast<float4 *>(dst + 4 * ((p / 2) ^ s)) = make_float4(v[p].x, v[p].y, v[p + 1].x, v[p + 1].y);
    } else {
        *reinterpret_cast<float2 *>(dst) = v[0];
    }
}

__device__ __forceinline__ float hsum(float2 v) { return v.x + v.y; }

// x rounded to TF32 (11 significant bits, nearest, ties away from zero), in an FP32 container
// whose low 13 mantissa bits are zero; x - tf32_rna(x) is exact in FP32
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int D>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int off = D / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Exact sum over the D lanes of a chain as an unevaluated pair hi + lo (TwoSum at every level).
template <int D>
__device__ __forceinline__ void group_sum_exact(float v, float &hi, float &lo) {
    float err = 0.0f;
#pragma unroll
    for (int off = D / 2; off > 0; off >>= 1) {
        const float pv = __shfl_xor_sync(0xffffffffu, v, off);
        const float pe = __shfl_xor_sync(0xffffffffu, err, off);
        // both partners form the same sum: order the operands by lane so they round alike
        const bool low = (threadIdx.x & off) == 0;
        const float x = low ? v : pv, y = low ? pv : v;
        const float sum = x + y;
        const float bb = sum - x;
        const float e = (x - (sum - bb)) + (y - bb);
        err = (low ? err + pe : pe + err) + e;
        v = sum;
    }
    hi = v;
    lo = err;
}

// q^dag p for the lane's own column q = (qr, qi) (pairs of rows, in registers) and a column p
// in shared memory (real and imaginary planes), without rounding error in the products and
// the sum: each product is accumulated into s1, which carries the offset `offset` = 1.5 2^(e+1)
// and so holds its running sum rounded to multiples of 2^(e-22) exactly (every partial sum of
// one accumulator must stay below 2^e); the FMA's rounding error x y - (s1' - s1) is formed
// exactly by a second FMA and summed in s2, where it is at most 2^(e-23).  The result is
// returned as (re, im), minus `sub` on the real part (subtracted while the sum is still
// exact); its error is about 2^(e-45) per product.
template <int D>
__device__ __forceinline__ float2 sum_products_exact(const float2 (&qr)[D / 2], const float2 (&qi)[D / 2],
                                                     const float *pre, const float *pim, float offset, float sub,
                                                     int s = 0) {
    // four accumulators: qr pr + qi pi (real part), qr pi and qi pr (imaginary part, subtracted
    // at the end); each a grid sum s1 and an error sum s2
    float2 a1 = make_float2(offset, offset), b1 = a1, c1 = a1;
    float2 a2 = make_float2(0.f, 0.f), b2 = a2, c2 = a2;
    auto step = [](float2 &s1, float2 &s2, float2 x, float2 y) {
        const float2 n = __ffma2_rn(x, y, s1);
        s2 = __fadd2_rn(s2, __ffma2_rn(x, y, sub2(s1, n)));   // + (x y - (n - s1)): the rounding error
        s1 = n;
    };
    // the column p is read two row pairs (one 128-bit load per plane) at a time
#pragma unroll
    for (int p0 = 0; p0 < D / 2; p0 += (D >= 4 ? 2 : 1)) {
        float2 pr[2], pi[2];
        if constexpr (D >= 4) {
            const float4 r4 = *reinterpret_cast<const float4 *>(pre + 4 * ((p0 / 2) ^ s));   // (block swizzle s)
            const float4 i4 = *reinterpret_cast<const float4 *>(pim + 4 * ((p0 / 2) ^ s));
            pr[0] = make_float2(r4.x, r4.y);
            pr[1] = make_float2(r4.z, r4.w);
            pi[0] = make_float2(i4.x, i4.y);
            pi[1] = make_float2(i4.z, i4.w);
        } else {
            pr[0] = *reinterpret_cast<const float2 *>(pre);
            pi[0] = *reinterpret_cast<const float2 *>(pim);
        }
#pragma unroll
        for (int u = 0; u < (D >= 4 ? 2 : 1); ++u) {
            const int p = p0 + u;
            step(a1, a2, qr[p], pr[u]);   // Re: qr pr + qi pi
            step(a1, a2, qi[p], pi[u]);
            step(b1, b2, qr[p], pi[u]);   // Im: qr pi - qi pr
            step(c1, c2, qi[p], pr[u]);
        }
    }
    // the grid parts minus their offsets are exact, and so are their sums and differences
    const float re_grid = ((a1.x - offset) + (a1.y - offset)) - sub;
    const float im_grid = ((b1.x - offset) + (b1.y - offset)) - ((c1.x - offset) + (c1.y - offset));
    return make_float2(re_grid + (a2.x + a2.y), im_grid + ((b2.x + b2.y) - (c2.x + c2.y)));
}

struct ProposeArgs {
    const float *x_eval;        // MODE_EVAL: [rows][nx] latent vectors
    float *y;                   // [2][R][nx]
    const uint8_t *cur;         // [R]
    const float2 *coef;         // [R] (sqrt(1 - beta^2), beta) as floats
    float *rho_out;             // [rows][d_pad] packed rho (FP32-normalised)
    __nv_bfloat16 *split_out;   // [rows][3][d_pad] bf16 hi/mid/lo, or null
    float *split_tf;            // [rows][tf_splits][d_pad] TF32 hi[, lo], or null
    int tf_splits;              // 1 or 2
    double *trace_out;          // [rows] exact trace of the stored rho (1 up to rounding)
    float *rho_norm_out;        // MODE_EVAL, optional: [rows][d] copy of the packed rho
    int64_t rows;
    int64_t R;
    int64_t chain_offset;
    uint64_t seed;
    uint32_t step;
    const StepState *step_dev;   // MODE_STEP: when not null the step is read from here
    int mode;
    int d_pad;
    Philox::RoundKeys rk;        // the generator's round keys for `seed`
};

// The rest of a refinement pass at D >= 32 (the solve, Y's upper part and diagonal, U = Q1 -
// Q1 Y^dag), with rolled loops and Y's row j kept in place in area B: unrolled over registers, as
// refine_pass does for D <= 16, the pass is several thousand straight-line instructions at D = 32
// and the warps stall on instruction fetch.  The arithmetic of each entry is refine_pass's.  Lane j
// writes only row j of area B: its lower part (read by the other lanes for their upper parts only
// after the barrier below), then its diagonal and upper part, which no other lane reads.
template <int D, int QC>
__device__ __noinline__ float refine_tail_rolled(float *qre, float *qim, float *hre, float *him, const float2 *rpk,
                                                 int j, float2 mjj, bool apply) {
    auto cidx = [](int r, int cc) { return cc * D + (r ^ cc); };
    // forward substitution on row j: entries c < j only (the row has no unknowns beyond)
#pragma unroll 1
    for (int c0 = 0; c0 < j; ++c0) {
        const float inv_r = rpk[c0 * (c0 + 1) / 2 + c0].y;
        const int o0 = cidx(j, c0);
        const float ar = hre[o0] * inv_r, ai = him[o0] * inv_r;
        hre[o0] = ar;
        him[o0] = ai;
#pragma unroll 2
        for (int c = c0 + 1; c < j; ++c) {
            const float2 r = rpk[c * (c + 1) / 2 + c0];   // R[c0][c]
            const int o = cidx(j, c);
            hre[o] -= ar * r.x - ai * r.y;
            him[o] -= ar * r.y + ai * r.x;
        }
    }
    // diagonal: Re Y_jj = (N_jj - 1) / 2; Im Y_jj makes R_jj real
    float ydi = mjj.y;
    float ymax = 0.0f;
#pragma unroll 1
    for (int k = 0; k < j; ++k) {
        const float2 r = rpk[j * (j + 1) / 2 + k];   // R[k][j]
        const float yr = hre[cidx(j, k)], yi = him[cidx(j, k)];
        ydi -= yr * r.y + yi * r.x;
        ymax = fmaxf(ymax, fmaxf(fabsf(yr), fabsf(yi)));
    }
    const float2 ydiag = make_float2(0.5f * hre[cidx(j, j)], ydi * rpk[j * (j + 1) / 2 + j].y);
    __syncwarp();   // every lane's lower row is in place
    // upper part: Y[j][c] = N_jc - conj(Y[c][j]), c > j, over N_jc; every lane walks the same c
    // (its entries (j, c) and (c, j) then lie in distinct banks across the lanes)
#pragma unroll 2
    for (int c = 1; c < D; ++c) {
        if (c > j) {
            const float yr = hre[cidx(j, c)] - hre[cidx(c, j)], yi = him[cidx(j, c)] + him[cidx(c, j)];
            hre[cidx(j, c)] = yr;
            him[cidx(j, c)] = yi;
            ymax = fmaxf(ymax, fmaxf(fabsf(yr), fabsf(yi)));
        }
    }
    hre[cidx(j, j)] = ydiag.x;
    him[cidx(j, j)] = ydiag.y;
    ymax = fmaxf(ymax, fmaxf(fabsf(ydiag.x), fabsf(ydiag.y)));
#pragma unroll
    for (int off = D / 2; off >= 1; off /= 2) ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, off, D));
    // U = Q1 - Q1 Y^dag: column j is q_j - sum_k q_k conj(Y[j][k]), in two halves of rows as in
    // refine_pass
    constexpr int HP = D / 4;   // row pairs per half
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        float2 cr[HP], ci[HP];
#pragma unroll
        for (int p = 0; p < HP; ++p) cr[p] = ci[p] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int k = 0; k < D; ++k) {
            const float ykr = hre[cidx(j, k)], yki = him[cidx(j, k)];
            const float2 yx = make_float2(ykr, ykr), yy = make_float2(yki, yki), myy = make_float2(-yki, -yki);
#pragma unroll
            for (int p = 0; p < HP; p += 2) {   // (vr + i vi)(y.x - i y.y), a 4-float block of rows at a time
                const int o = k * QC + 2 * (half * HP + p);
                const float4 r4 = *reinterpret_cast<const float4 *>(qre + o);
                const float4 i4 = *reinterpret_cast<const float4 *>(qim + o);
                const float2 vr[2] = {make_float2(r4.x, r4.y), make_float2(r4.z, r4.w)};
                const float2 vi[2] = {make_float2(i4.x, i4.y), make_float2(i4.z, i4.w)};
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    cr[p + u] = __ffma2_rn(vr[u], yx, __ffma2_rn(vi[u], yy, cr[p + u]));
                    ci[p + u] = __ffma2_rn(vi[u], yx, __ffma2_rn(vr[u], myy, ci[p + u]));
                }
            }
        }
        __syncwarp();   // every lane has read this half of every q_k
        if (apply) {
#pragma unroll
            for (int p = 0; p < HP; p += 2) {
                const int o = j * QC + 2 * (half * HP + p);
                float4 *ur = reinterpret_cast<float4 *>(qre + o);
                float4 *ui = reinterpret_cast<float4 *>(qim + o);
                const float4 u0 = *ur, u1 = *ui;
                const float2 a0 = sub2(make_float2(u0.x, u0.y), cr[p]), a1 = sub2(make_float2(u0.z, u0.w), cr[p + 1]);
                const float2 b0 = sub2(make_float2(u1.x, u1.y), ci[p]), b1 = sub2(make_float2(u1.z, u1.w), ci[p + 1]);
                *ur = make_float4(a0.x, a0.y, a1.x, a1.y);
                *ui = make_float4(b0.x, b0.y, b1.x, b1.y);
            }
        }
        __syncwarp();
    }
    return ymax;
}

// One first-order pass of the refinement of U (step 2b of the D <= 16 kernel below, where the
// method is described).  `again`: a pass after the first, which reads H's column j back from y'
// into area B (it held C) and U's column j as this lane's vector; `apply`: write the refined U
// (a further pass runs for the whole warp when any of its chains needs it, and the others
// discard theirs, so a chain's bits never depend on its neighbours).  Returns the chain's
// largest |Y| entry.
template <int D, int QC>
__device__ __forceinline__ float refine_pass(float2 (&hr)[D / 2], float2 (&hi)[D / 2], float *qre, float *qim,
                                             float *hre, float *him, const float2 *rpk, const float *gsrc, int j,
                                             bool again, bool apply) {
    constexpr int d = D * D;
    auto cidx = [](int r, int cc) { return cc * D + (r ^ cc); };
    if (again) {   // H's column j into area B again (it held C), U's column j as the vector
#pragma unroll
        for (int i = 0; i < D; i += (D >= 4 ? 4 : 1)) {
            if constexpr (D >= 4) {
                const int o = j * D + 4 * ((i / 4) ^ hsw<D, QC>(j));
                *reinterpret_cast<float4 *>(hre + o) = *reinterpret_cast<const float4 *>(gsrc + 2 * d + j * D + i);
                *reinterpret_cast<float4 *>(him + o) = *reinterpret_cast<const float4 *>(gsrc + 3 * d + j * D + i);
            } else {
                hre[j * D + i] = gsrc[2 * d + j * D + i];
                him[j * D + i] = gsrc[3 * d + j * D + i];
            }
        }
        load_column2<D>(qre + j * QC, hr, qsw<D, QC>(j));
        load_column2<D>(qim + j * QC, hi, qsw<D, QC>(j));
        __syncwarp();
    }
#pragma unroll 1
    for (int cc = 0; cc < D; ++cc) {
        const bool lower = cc < j;   // M_jc = q_j^dag h_c; at c = j (and above) N_jc = q_j^dag q_c
        const float *pre = lower ? hre + cc * D : qre + cc * QC;
        const float *pim = lower ? him + cc * D : qim + cc * QC;
        // every partial sum of M stays below 2^6 (|h| < 64), of N below 2^1
        const float2 res = sum_products_exact<D>(hr, hi, pre, pim, lower ? 192.0f : 6.0f, cc == j ? 1.0f : 0.0f,
                                                 lower ? hsw<D, QC>(cc) : qsw<D, QC>(cc));
        __syncwarp();   // every lane is done with column c of H
        hre[cidx(j, cc)] = res.x;
        him[cidx(j, cc)] = res.y;
    }
    // M_jj, the one entry of the row not formed above: its column of H now holds C, so h_j is
    // read again from the proposal's own y' (or the evaluated row; for an inactive lane the
    // first chain's row, in bounds, whose result is not used)
    const float2 mjj = sum_products_exact<D>(hr, hi, gsrc + 2 * d + j * D, gsrc + 3 * d + j * D, 192.0f, 0.0f);
    __syncwarp();
    if constexpr (D >= 32) return refine_tail_rolled<D, QC>(qre, qim, hre, him, rpk, j, mjj, apply);
    // Y, row j, in registers: y[c] = Y[j][c].  Forward substitution, right-looking: after
    // Y[j][c0] = (M_jc0 - ...) / R_c0c0 every later entry of the row takes its share
    // -Y[j][c0] R[c0][c] at once, so each R entry is read once for all lanes; entries at
    // c >= j stay zero (the lane's row has no such unknowns) until the upper part below.
    float2 y[D];
#pragma unroll
    for (int c = 0; c < D; ++c)
        y[c] = (c < j) ? make_float2(hre[cidx(j, c)], him[cidx(j, c)]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int c0 = 0; c0 < D - 1; ++c0) {
        const float inv_r = rpk[c0 * (c0 + 1) / 2 + c0].y;
        y[c0] = make_float2(y[c0].x * inv_r, y[c0].y * inv_r);
#pragma unroll
        for (int c = c0 + 1; c < D - 1; ++c) {
            const float2 r = rpk[c * (c + 1) / 2 + c0];   // R[c0][c]
            y[c].x -= y[c0].x * r.x - y[c0].y * r.y;
            y[c].y -= y[c0].x * r.y + y[c0].y * r.x;
        }
    }
    // diagonal: Re Y_jj = (N_jj - 1) / 2; Im Y_jj makes R_jj real
    float ydi = mjj.y;
#pragma unroll
    for (int k = 0; k < D - 1; ++k) {
        const float2 r = rpk[j * (j + 1) / 2 + (k < j ? k : 0)];   // R[k][j] (k < j)
        if (k < j) ydi -= y[k].x * r.y + y[k].y * r.x;
    }
    const float2 ydiag = make_float2(0.5f * hre[cidx(j, j)], ydi * rpk[j * (j + 1) / 2 + j].y);
    // upper part: Y[j][c] = N_jc - conj(Y[c][j]), c > j, through area B
#pragma unroll
    for (int c = 0; c < D - 1; ++c)
        if (c < j) {
            hre[cidx(j, c)] = y[c].x;
            him[cidx(j, c)] = y[c].y;
        }
    __syncwarp();   // every lane's lower row is in place
#pragma unroll
    for (int c = 1; c < D; ++c)
        if (c > j) y[c] = make_float2(hre[cidx(j, c)] - hre[cidx(c, j)], him[cidx(j, c)] + him[cidx(c, j)]);
#pragma unroll
    for (int c = 0; c < D; ++c)
        if (c == j) y[c] = ydiag;
    // the chain's largest |Y| entry decides whether another pass follows
    float ymax = 0.0f;
#pragma unroll
    for (int c = 0; c < D; ++c) ymax = fmaxf(ymax, fmaxf(fabsf(y[c].x), fabsf(y[c].y)));
#pragma unroll
    for (int off = D / 2; off >= 1; off /= 2) ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, off, D));
    // U = Q1 - Q1 Y^dag: column j is q_j - sum_k q_k conj(Y[j][k]); the correction is summed
    // on its own (it is small) and subtracted once.  Rows go in two halves: a half is
    // overwritten only after every lane has read that half of every column.
    constexpr int HP = (D >= 4) ? D / 4 : 1;   // row pairs per half
#pragma unroll
    for (int half = 0; half < (D >= 4 ? 2 : 1); ++half) {
        float2 cr[HP], ci[HP];
#pragma unroll
        for (int p = 0; p < HP; ++p) cr[p] = ci[p] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float2 yx = make_float2(y[k].x, y[k].x), yy = make_float2(y[k].y, y[k].y);
            const float2 myy = make_float2(-y[k].y, -y[k].y);   // conj(y) = (y.x, -y.y)
            if constexpr (HP % 2 == 0) {   // column k's rows read a 4-float block (two pairs) at a time
#pragma unroll
                for (int p = 0; p < HP; p += 2) {   // (vr + i vi)(y.x - i y.y)
                    const int row = 2 * (half * HP + p);
                    const int o = k * QC + 4 * ((row >> 2) ^ qsw<D, QC>(k));
                    const float4 r4 = *reinterpret_cast<const float4 *>(qre + o);
                    const float4 i4 = *reinterpret_cast<const float4 *>(qim + o);
                    const float2 vr[2] = {make_float2(r4.x, r4.y), make_float2(r4.z, r4.w)};
                    const float2 vi[2] = {make_float2(i4.x, i4.y), make_float2(i4.z, i4.w)};
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        cr[p + u] = __ffma2_rn(vr[u], yx, __ffma2_rn(vi[u], yy, cr[p + u]));
                        ci[p + u] = __ffma2_rn(vi[u], yx, __ffma2_rn(vr[u], myy, ci[p + u]));
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < HP; ++p) {   // (vr + i vi)(y.x - i y.y)
                    const int row = 2 * (half * HP + p);
                    const int o = k * QC + 4 * ((row >> 2) ^ qsw<D, QC>(k)) + (row & 3);
                    const float2 vr = *reinterpret_cast<const float2 *>(qre + o);
                    const float2 vi = *reinterpret_cast<const float2 *>(qim + o);
                    cr[p] = __ffma2_rn(vr, yx, __ffma2_rn(vi, yy, cr[p]));
                    ci[p] = __ffma2_rn(vi, yx, __ffma2_rn(vr, myy, ci[p]));
                }
            }
        }
        __syncwarp();   // every lane has read this half of every q_k
        if (apply) {
            if constexpr (HP % 2 == 0) {   // two row pairs, one 4-float block, at a time
#pragma unroll
                for (int p = 0; p < HP; p += 2) {
                    const int row = 2 * (half * HP + p);
                    float4 *ur = reinterpret_cast<float4 *>(qre + j * QC + 4 * ((row >> 2) ^ qsw<D, QC>(j)));
                    float4 *ui = reinterpret_cast<float4 *>(qim + j * QC + 4 * ((row >> 2) ^ qsw<D, QC>(j)));
                    const float4 u0 = *ur, u1 = *ui;
                    const float2 a0 = sub2(make_float2(u0.x, u0.y), cr[p]), a1 = sub2(make_float2(u0.z, u0.w), cr[p + 1]);
                    const float2 b0 = sub2(make_float2(u1.x, u1.y), ci[p]), b1 = sub2(make_float2(u1.z, u1.w), ci[p + 1]);
                    *ur = make_float4(a0.x, a0.y, a1.x, a1.y);
                    *ui = make_float4(b0.x, b0.y, b1.x, b1.y);
                }
            } else {
#pragma unroll
                for (int p = 0; p < HP; ++p) {
                    const int row = 2 * (half * HP + p);
                    float2 *ur = reinterpret_cast<float2 *>(qre + j * QC + row);
                    float2 *ui = reinterpret_cast<float2 *>(qim + j * QC + row);
                    *ur = sub2(*ur, cr[p]);
                    *ui = sub2(*ui, ci[p]);
                }
            }
        }
        __syncwarp();
    }
    return ymax;
}

// The passes after the first, for the few chains whose first pass left |Y| above kRefineTol: out
// of line, so that the common path keeps its registers.
template <int D, int QC>
__device__ __noinline__ void refine_more(float *qre, float *qim, float *hre, float *him, const float2 *rpk,
                                         const float *gsrc, int j, float ymax) {
    float2 hr[D / 2], hi[D / 2];
#pragma unroll 1
    for (int pass = 1; pass < kRefinePasses && __any_sync(0xffffffffu, ymax > kRefineTol); ++pass) {
        const bool need = ymax > kRefineTol;
        const float next = refine_pass<D, QC>(hr, hi, qre, qim, hre, him, rpk, gsrc, j, true, need);
        ymax = need ? next : ymax;
    }
}

// THREADS: the CTA size (chains per CTA = THREADS / D); 128 by default, 64 or 32 when the
// autotuner finds that a small problem covers more SMs that way.  The register budget per
// thread is the same for every size (five 128-thread CTAs' worth per SM).
template <int D, int PASSES, int THREADS = kThreads>
__global__ void __launch_bounds__(THREADS, 5 * kThreads / THREADS) propose_kernel(ProposeArgs a) {
    using S = Shape<D, PASSES, THREADS>;
    constexpr int d = S::d;
    constexpr int nx = 4 * d;
    constexpr int RS = S::row_stride;
    constexpr int QC = S::qcol;
    constexpr int PK = S::pk_stride;
    extern __shared__ __align__(16) float smem[];

    const int j = threadIdx.x % D;       // owned column (and, in steps 2b and 4, owned row)
    const int g = threadIdx.x / D;       // chain slot in the block
    const int64_t c = (int64_t)blockIdx.x * S::chains_per_block + g;
    const bool active = c < a.rows;
    const uint32_t step = (a.step_dev && a.mode == MODE_STEP) ? a.step_dev->step : a.step;
    float *sm = smem + g * S::smem_floats;
    float *qre = sm, *qim = sm + D * QC;                 // Q planes (column stride QC)
    float2 *wsm = reinterpret_cast<float2 *>(sm);        // W row-major (row stride RS), replaces Q
    float *fre = sm + S::area_a, *fim = fre + D * D;     // F column-major (stride D), re / im planes
    float *packed = sm + S::area_a;                      // staged rho (row stride PK), replaces F
    float *hre = sm + S::area_a, *him = hre + D * D;     // PASSES = 3: H's columns (stride D), in area B
    float2 *rpk = reinterpret_cast<float2 *>(sm + S::area_a + S::area_b);   // PASSES = 3: packed R

    // ---- 1. latent proposal --------------------------------------------------------------
    float coef_y = 1.0f, coef_eta = 0.0f;
    int cur = 0;
    if (active && a.mode == MODE_STEP) {
        cur = a.cur[c];
        const float2 cf = a.coef[c];
        coef_y = cf.x;
        coef_eta = cf.y;
    } else if (a.mode == MODE_INIT) {
        coef_y = 0.0f;
        coef_eta = 1.0f;
    }
    const int64_t cc = active ? c : 0;
    const uint32_t chain_id = (uint32_t)(a.chain_offset + cc);
    const uint32_t tag = (a.mode == MODE_INIT) ? TAG_INIT : TAG_PROPOSAL;
    const float *ysrc = a.y + ((int64_t)cur * a.R + cc) * nx;
    float *ydst = a.y + ((int64_t)(1 - cur) * a.R + cc) * nx;
    // where G's column j is read back in step 3: this lane's own y' writes, or the input row
    const float *gsrc = (a.mode == MODE_EVAL) ? a.x_eval + cc * nx : ydst;
    float2 hr[D / 2], hi[D / 2];   // H's column j, entries (2p, 2p + 1) in pair p
    if constexpr (D >= 4) {
        // lane j owns entries j D .. j D + D - 1 of each part: D/4 Philox blocks per part
#pragma unroll 1
        for (int part = 0; part < 4; ++part) {
            const int e0 = part * d + j * D;    // element index of (row 0, column j)
            float4 y0[D / 4];
#pragma unroll
            for (int q = 0; q < D / 4; ++q) {
                y0[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (active && a.mode == MODE_STEP) y0[q] = *reinterpret_cast<const float4 *>(ysrc + e0 + 4 * q);
                if (active && a.mode == MODE_EVAL) y0[q] = *reinterpret_cast<const float4 *>(a.x_eval + cc * nx + e0 + 4 * q);
            }
#pragma unroll
            for (int q = 0; q < D / 4; ++q) {
                float4 yn = y0[q];
                if (a.mode != MODE_EVAL) {
                    const uint4 w = Philox::block(make_uint4((uint32_t)(e0 / 4 + q), step, chain_id, tag), a.rk);
                    float z0, z1, z2, z3;
                    gaussian_pair_fast(w.x, w.y, z0, z1);
                    gaussian_pair_fast(w.z, w.w, z2, z3);
                    yn.x = __fmaf_rn(coef_y, y0[q].x, coef_eta * z0);
                    yn.y = __fmaf_rn(coef_y, y0[q].y, coef_eta * z1);
                    yn.z = __fmaf_rn(coef_y, y0[q].z, coef_eta * z2);
                    yn.w = __fmaf_rn(coef_y, y0[q].w, coef_eta * z3);
                    if (active) *reinterpret_cast<float4 *>(ydst + e0 + 4 * q) = yn;
                }
                if (part == 2) {
                    hr[2 * q] = make_float2(yn.x, yn.y);
                    hr[2 * q + 1] = make_float2(yn.z, yn.w);
                } else if (part == 3) {
                    hi[2 * q] = make_float2(yn.x, yn.y);
                    hi[2 * q + 1] = make_float2(yn.z, yn.w);
                }
            }
        }
    } else {
        // D == 2: each part is one Philox block shared by the two lanes; lane j takes pair j
#pragma unroll
        for (int part = 0; part < 4; ++part) {
            const int e = part * d + j * D;
            float y0v = 0.0f, y1v = 0.0f;
            if (a.mode == MODE_EVAL) {
                if (active) {
                    y0v = a.x_eval[cc * nx + e];
                    y1v = a.x_eval[cc * nx + e + 1];
                }
            } else {
                const uint4 w = Philox::block(make_uint4((uint32_t)part, step, chain_id, tag), a.rk);
                float z0, z1;
                gaussian_pair_fast(j == 0 ? w.x : w.z, j == 0 ? w.y : w.w, z0, z1);
                float o0 = 0.0f, o1 = 0.0f;
                if (a.mode == MODE_STEP && active) {
                    o0 = ysrc[e];
                    o1 = ysrc[e + 1];
                }
                y0v = __fmaf_rn(coef_y, o0, coef_eta * z0);
                y1v = __fmaf_rn(coef_y, o1, coef_eta * z1);
                if (active) {
                    ydst[e] = y0v;
                    ydst[e + 1] = y1v;
                }
            }
            if (part == 2) {
                hr[0] = make_float2(y0v, y1v);
            } else if (part == 3) {
                hi[0] = make_float2(y0v, y1v);
            }
        }
    }

    if constexpr (PASSES == 3) {   // H's original columns, for the refinement after the sweep
        store_column2<D>(hre + j * D, hr, hsw<D, QC>(j));
        store_column2<D>(him + j * D, hi, hsw<D, QC>(j));
    }

    // ---- 2a. modified Gram-Schmidt on the columns of H (Algorithm 1) ---------------------------
    // Every lane loads the published column v_k and forms r = v_k^dag h with its own column h
    // (packed f32x2 products over pairs of rows).  Lane k's column is v_k itself, so its r is
    // |v_k|^2, which the other lanes take by shuffle.  Lanes j > k project; lane k keeps
    // 1/|v_k|; a lane j < k holds its final v_j, so its r is conj(v_j^dag v_k) and gives the
    // Gram entry E_jk = q_j^dag q_k of the normalised columns for the re-orthogonalisation --
    // the entries become available exactly as lanes fall idle, so the Gram matrix costs no
    // separate pass.
    // PASSES = 0 (the Hilbert-Schmidt prior) skips steps 2 and the U term of step 3: W = G
    if constexpr (PASSES > 0) {
    float inv_own = 0.0f;   // 1 / |v_j| of this lane's final column
#pragma unroll 1
    for (int k = 0; k < D; ++k) {
        if (j == k) {   // column k is final: publish it
            store_column2<D>(qre + k * QC, hr, qsw<D, QC>(k));
            store_column2<D>(qim + k * QC, hi, qsw<D, QC>(k));
        }
        __syncwarp();
        float2 vr[D / 2], vi[D / 2];
        load_column2<D>(qre + k * QC, vr, qsw<D, QC>(k));
        load_column2<D>(qim + k * QC, vi, qsw<D, QC>(k));
        // r = v^dag h = sum (vr hr + vi hi) + i sum (vr hi - vi hr)
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
        for (int p = 0; p < D / 2; ++p) {
            a0 = __ffma2_rn(vr[p], hr[p], a0);
            a1 = __ffma2_rn(vi[p], hi[p], a1);
            b0 = __ffma2_rn(vr[p], hi[p], b0);
            b1 = __ffma2_rn(vi[p], hr[p], b1);
        }
        const float rr = hsum(a0) + hsum(a1);
        const float ri = hsum(b0) - hsum(b1);
        const float nk = __shfl_sync(0xffffffffu, rr, k, D);   // |v_k|^2 from lane k
        // one hardware reciprocal square root, uniform over the lanes: its few-ulp error in the
        // projection coefficient or the norm is of the size of the FP32 rounding the sweep
        // already leaves, and the re-orthogonalisation removes both to first order
        const float rs = rsqrtf(nk);
        // h -= (r / |v|^2) v on lanes j > k; the coefficient is zero elsewhere, which leaves h
        // unchanged, so the warp runs one branch-free path
        const float coef = (j > k) ? rs * rs : 0.0f;
        const float sr = rr * coef, si = ri * coef;
        const float2 msr = make_float2(-sr, -sr), psi = make_float2(si, si), msi = make_float2(-si, -si);
#pragma unroll
        for (int p = 0; p < D / 2; ++p) {
            hr[p] = __ffma2_rn(msr, vr[p], __ffma2_rn(psi, vi[p], hr[p]));
            hi[p] = __ffma2_rn(msr, vi[p], __ffma2_rn(msi, vr[p], hi[p]));
        }
        inv_own = (j == k) ? rs : inv_own;
        if constexpr (PASSES == 2) {
            if (j < k) {
                const float sc = inv_own * rs;             // E_jk = conj(r) / (|v_j| |v_k|), j < k
                fre[k * D + j] = rr * sc;
                fim[k * D + j] = -ri * sc;
            }
        }
        if constexpr (PASSES == 3) {
            // the triangular factor the refinement solves with (FP32 suffices there): R_kj =
            // v_k^dag h_j / |v_k| above the diagonal; the diagonal slot holds (|v_k|, 1 / |v_k|)
            if (j > k) rpk[j * (j + 1) / 2 + k] = make_float2(rr * rs, ri * rs);
            if (j == k) rpk[k * (k + 1) / 2 + k] = make_float2(nk * rs, rs);
        }
    }
    {   // normalise the own column and publish it
        const float2 sc = make_float2(inv_own, inv_own);
#pragma unroll
        for (int p = 0; p < D / 2; ++p) {
            hr[p] = __fmul2_rn(hr[p], sc);
            hi[p] = __fmul2_rn(hi[p], sc);
        }
        __syncwarp();
        store_column2<D>(qre + j * QC, hr, qsw<D, QC>(j));
        store_column2<D>(qim + j * QC, hi, qsw<D, QC>(j));
        __syncwarp();
    }
    }   // PASSES > 0

    if constexpr (PASSES == 3) {
        // ---- 2b. refinement of Q1 to the QR factor of H beyond FP32 ----------------------------
        // An FP32 Gram-Schmidt factor Q1 is the exact factor of a matrix within 2^-24 of H, so it
        // misses U by about cond(H) 2^-24 -- and near the posterior U + I is nearly singular, so
        // that error reaches rho.  With Q1 = U V, V = I + X small: N = Q1^dag Q1 = I + X + X^dag
        // (first order) and M = Q1^dag H = V^dag R, whose strictly lower part is that of X^dag R.
        // So X^dag (called Y below) has: strictly lower part from the triangular system
        // lower(Y R) = lower(M), upper part N - conj(lower part)^T, real diagonal (N_jj - 1) / 2,
        // imaginary diagonal from the real diagonal of R; and U = Q1 V^-1 = Q1 (I - Y^dag) to
        // first order.  The step leaves about |Y|^2 (|Y| ~ cond(H) 2^-24): below FP32 rounding
        // while every |Y| entry is below 2^-14 (cond(H) up to ~10^3).  A chain above that repeats
        // the step from the refined U, its H and the same R; each pass squares the residual, and
        // three passes cover cond(H) up to ~10^6.  (The posterior's chains reach cond(H) ~10^5:
        // one chain in 1024 of a four-qubit problem with 81,000 shots after 2000 steps, which a
        // single pass left 6e-3 from the oracle's log L.)
        // The lower part of M and N - I are tiny differences of O(1) products, so they are formed
        // without rounding error: lane j forms row j (c < j: M_jc = q_j^dag h_c; c > j: N_jc =
        // q_j^dag q_c) with error-free products (sum_products_exact), its own q_j in (hr, hi) and
        // the other vector read from shared memory -- the lanes take different vectors at the
        // same step only through their addresses, so every lane does useful work at every step.
        // Lanes c > j then solve row j of the lower system as M_jc arrives (R from the sweep).
        // C[j][c] (row j = lane j) is kept in area B: step c frees H's column c, whose 2 D floats
        // take the D lanes' results of that step -- element (r, c) at c D + (r ^ c) of the real
        // (hre) and imaginary (him) planes, so that the lanes' writes of a step, a lane's reads
        // of its row and the reads of a column all hit distinct banks.
        const float ymax = refine_pass<D, QC>(hr, hi, qre, qim, hre, him, rpk, gsrc, j, false, true);
        if (__any_sync(0xffffffffu, ymax > kRefineTol)) refine_more<D, QC>(qre, qim, hre, him, rpk, gsrc, j, ymax);
    }

    if constexpr (PASSES == 2) {
        // ---- 2b. re-orthogonalisation Q2 = Q1 (I - F), F = strict upper part of E (formed in
        // the sweep above) plus half the diagonal E_jj = |q_j|^2 - 1 of the stored columns ------
        {
            float2 n = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < D / 2; ++p) n = __ffma2_rn(hr[p], hr[p], __ffma2_rn(hi[p], hi[p], n));
            fre[j * D + j] = 0.5f * (hsum(n) - 1.0f);
            fim[j * D + j] = 0.0f;
            if (j + 1 < D) {   // F[j+1][j] = 0: read in the pair (j, j+1) of column j
                fre[j * D + j + 1] = 0.0f;
                fim[j * D + j + 1] = 0.0f;
            }
        }
        __syncwarp();
        // row a of Q2: x_m - sum_{i <= m} x_i F[i][m], x = row a of Q1 (lane a = j), as pairs
        // (x_2p, x_2p+1); a pair that reaches past m meets F[m+1][m] = 0
        {
            float2 xr[D / 2], xi[D / 2];
#pragma unroll
            for (int p = 0; p < D / 2; ++p) {
                xr[p] = make_float2(qre[(2 * p) * QC + j], qre[(2 * p + 1) * QC + j]);
                xi[p] = make_float2(qim[(2 * p) * QC + j], qim[(2 * p + 1) * QC + j]);
            }
#pragma unroll
            for (int m = D - 1; m >= 0; --m) {   // descending: x_m is still Q1's when row m is formed
                float2 ca = make_float2(0.f, 0.f), cb = ca, cc2 = ca, cd = ca;
#pragma unroll
                for (int p = 0; 2 * p <= m; ++p) {
                    float2 fx, fy;   // F[2p][m], F[2p+1][m]
                    if constexpr (D >= 4) {
                        if ((p & 1) == 0) {
                            const float4 f4x = *reinterpret_cast<const float4 *>(fre + m * D + 2 * p);
                            const float4 f4y = *reinterpret_cast<const float4 *>(fim + m * D + 2 * p);
                            fx = make_float2(f4x.x, f4x.y);
                            fy = make_float2(f4y.x, f4y.y);
                        } else {
                            fx = *reinterpret_cast<const float2 *>(fre + m * D + 2 * p);
                            fy = *reinterpret_cast<const float2 *>(fim + m * D + 2 * p);
                        }
                    } else {
                        fx = *reinterpret_cast<const float2 *>(fre + m * D + 2 * p);
                        fy = *reinterpret_cast<const float2 *>(fim + m * D + 2 * p);
                    }
                    ca = __ffma2_rn(xr[p], fx, ca);    // sum xr fx
                    cb = __ffma2_rn(xi[p], fy, cb);    // sum xi fy
                    cc2 = __ffma2_rn(xr[p], fy, cc2);  // sum xr fy
                    cd = __ffma2_rn(xi[p], fx, cd);    // sum xi fx
                }
                const float dr = hsum(ca) - hsum(cb), di = hsum(cc2) + hsum(cd);
                if (m & 1) {
                    xr[m / 2].y -= dr;
                    xi[m / 2].y -= di;
                } else {
                    xr[m / 2].x -= dr;
                    xi[m / 2].x -= di;
                }
            }
#pragma unroll
            for (int p = 0; p < D / 2; ++p) {
                qre[(2 * p) * QC + j] = xr[p].x;
                qre[(2 * p + 1) * QC + j] = xr[p].y;
                qim[(2 * p) * QC + j] = xi[p].x;
                qim[(2 * p + 1) * QC + j] = xi[p].y;
            }
        }
        __syncwarp();
    }

    if constexpr (D == 16) {
        // ---- 3. W = (U + I) G in 4x4 register blocks: lane (bi, bj) forms W[4bi.., 4bj..] -----
        // G is staged row-major as separate real and imaginary planes in area B (free between
        // the re-orthogonalisation and the packed rho), so that columns (4bj, 4bj+1) and
        // (4bj+2, 4bj+3) of a row are f32x2 pairs and U's entries enter broadcast: eight
        // packed FMAs per row of U instead of sixteen scalar ones.
        float *gsr = sm + S::area_a, *gsi = gsr + D * D;
        {
            float gr[D], gi[D];
            if (active) {
                load_column<D>(gsrc + j * D, gr);
                load_column<D>(gsrc + d + j * D, gi);
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i) gr[i] = gi[i] = 0.0f;
            }
#pragma unroll
            for (int i = 0; i < D; ++i) {
                gsr[i * D + j] = gr[i];
                gsi[i * D + j] = gi[i];
            }
        }
        __syncwarp();
        const int bi = j >> 2, bj = j & 3;
        // W[4bi + r][4bj + 2h .. 4bj + 2h + 1], two rows at a time: the products of Re U (and G
        // itself, the identity's term) in one pair of chains (wr, wi), those of Im U in another
        // (xr, xi), added at the end -- each chain half as long, with the rounding of the two
        // sums kept apart until the one final add (the assembly's log L error grows with the
        // length of the chains that form W).  The first two rows wait in registers until
        // every lane is done with U, whose storage W takes.
        float2 wr[4][2], wi[4][2];
#pragma unroll
        for (int hb = 0; hb < 2; ++hb) {
            float2 ar[2][2], ai[2][2], xr[2][2], xi[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int row = 4 * bi + 2 * hb + r;
                const float4 g4r = *reinterpret_cast<const float4 *>(gsr + row * D + 4 * bj);
                const float4 g4i = *reinterpret_cast<const float4 *>(gsi + row * D + 4 * bj);
                ar[r][0] = make_float2(g4r.x, g4r.y);
                ar[r][1] = make_float2(g4r.z, g4r.w);
                ai[r][0] = make_float2(g4i.x, g4i.y);
                ai[r][1] = make_float2(g4i.z, g4i.w);
                xr[r][0] = xr[r][1] = xi[r][0] = xi[r][1] = make_float2(0.f, 0.f);
            }
#pragma unroll 4
            for (int k = 0; k < (PASSES > 0 ? D : 0); ++k) {
                const float2 ur2 = *reinterpret_cast<const float2 *>(qre + k * QC + 4 * (bi ^ qsw<D, QC>(k)) + 2 * hb);
                const float2 ui2 = *reinterpret_cast<const float2 *>(qim + k * QC + 4 * (bi ^ qsw<D, QC>(k)) + 2 * hb);
                const float4 g4r = *reinterpret_cast<const float4 *>(gsr + k * D + 4 * bj);
                const float4 g4i = *reinterpret_cast<const float4 *>(gsi + k * D + 4 * bj);
                const float2 gr2[2] = {make_float2(g4r.x, g4r.y), make_float2(g4r.z, g4r.w)};
                const float2 gi2[2] = {make_float2(g4i.x, g4i.y), make_float2(g4i.z, g4i.w)};
                const float ur[2] = {ur2.x, ur2.y}, ui[2] = {ui2.x, ui2.y};
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float2 pu = make_float2(ur[r], ur[r]), pi = make_float2(ui[r], ui[r]);
                    const float2 mi = make_float2(-ui[r], -ui[r]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        ar[r][h] = __ffma2_rn(pu, gr2[h], ar[r][h]);
                        xr[r][h] = __ffma2_rn(mi, gi2[h], xr[r][h]);
                        ai[r][h] = __ffma2_rn(pu, gi2[h], ai[r][h]);
                        xi[r][h] = __ffma2_rn(pi, gr2[h], xi[r][h]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    wr[2 * hb + r][h] = __fadd2_rn(ar[r][h], xr[r][h]);
                    wi[2 * hb + r][h] = __fadd2_rn(ai[r][h], xi[r][h]);
                }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 4; ++r) {   // W row-major with padded rows (replaces Q)
            *reinterpret_cast<float4 *>(wsm + (4 * bi + r) * RS + 4 * bj) =
                make_float4(wr[r][0].x, wi[r][0].x, wr[r][0].y, wi[r][0].y);
            *reinterpret_cast<float4 *>(wsm + (4 * bi + r) * RS + 4 * bj + 2) =
                make_float4(wr[r][1].x, wi[r][1].x, wr[r][1].y, wi[r][1].y);
        }
        __syncwarp();
    } else {
    // ---- 3. W = (U + I) G, column j: W[:,j] = G[:,j] + sum_k U[:,k] G[k,j] ------------------
        float gr[D], gi[D], wr[D], wi[D];
        if (active) {
            load_column<D>(gsrc + j * D, gr);
            load_column<D>(gsrc + d + j * D, gi);
        } else {
    #pragma unroll
            for (int i = 0; i < D; ++i) {
                gr[i] = 0.0f;
                gi[i] = 0.0f;
            }
        }
    #pragma unroll
        for (int i = 0; i < D; ++i) {
            wr[i] = gr[i];
            wi[i] = gi[i];
        }
    #pragma unroll
        for (int k = 0; k < (PASSES > 0 ? D : 0); ++k) {
            float ur[D], ui[D];
            load_column<D>(qre + k * QC, ur, qsw<D, QC>(k));
            load_column<D>(qim + k * QC, ui, qsw<D, QC>(k));
    #pragma unroll
            for (int i = 0; i < D; ++i) {
                wr[i] = __fmaf_rn(ur[i], gr[k], __fmaf_rn(-ui[i], gi[k], wr[i]));
                wi[i] = __fmaf_rn(ur[i], gi[k], __fmaf_rn(ui[i], gr[k], wi[i]));
            }
        }
        __syncwarp();
        // W row-major with padded rows: W[i][j] at wsm[i * RS + j] (replaces Q)
    #pragma unroll
        for (int i = 0; i < D; ++i) wsm[i * RS + j] = make_float2(wr[i], wi[i]);
        __syncwarp();
    
    }

    // ---- 4. rho = W W^dag / Tr: lane a owns entries (a, a + t mod D), t = 0..D/2 ------------
    // (W W^dag)_ab = sum_m W[a,m] conj(W[b,m]): with the row of b read as complex pairs
    // (Re, Im) W[b,m], Re is the sum of both halves of (Re, Im) W[a,m] * (Re, Im) W[b,m] and Im
    // that of (Im, -Re) W[a,m] * (Re, Im) W[b,m]
    const int arow = j;
    float2 wa[D], wc[D];   // (Re, Im) W[a,m] and (Im, -Re) W[a,m]
#pragma unroll
    for (int m = 0; m < D; m += 2) {
        const float4 v = *reinterpret_cast<const float4 *>(wsm + arow * RS + m);
        wa[m] = make_float2(v.x, v.y);
        wa[m + 1] = make_float2(v.z, v.w);
        wc[m] = make_float2(v.y, -v.x);
        wc[m + 1] = make_float2(v.w, -v.z);
    }
    float diag;
    {
        float2 d0 = make_float2(0.f, 0.f), d1 = d0;
#pragma unroll
        for (int m = 0; m < D; m += 2) {
            d0 = __ffma2_rn(wa[m], wa[m], d0);
            d1 = __ffma2_rn(wa[m + 1], wa[m + 1], d1);
        }
        diag = hsum(d0) + hsum(d1);
    }
    const float inv_tr = 1.0f / group_sum<D>(diag);
    const float diag_n = diag * inv_tr;
    float tr_hi, tr_lo;
    group_sum_exact<D>(diag_n, tr_hi, tr_lo);   // exact trace of the stored diagonal
    packed[arow * PK + arow] = diag_n;
    // For t = D/2 lanes a and a + D/2 both form the entry pair {a, a + D/2}; the two results are
    // bitwise equal (the same products, accumulated in the same order, negated where the
    // conjugate is taken), so both stores may stand.
#pragma unroll 1
    for (int t = 1; t <= D / 2; ++t) {
        const int b = (arow + t) & (D - 1);
        float2 re0 = make_float2(0.f, 0.f), im0 = re0, re1 = re0, im1 = re0;
#pragma unroll
        for (int m = 0; m < D; m += 2) {
            const float4 wb = *reinterpret_cast<const float4 *>(wsm + b * RS + m);
            const float2 b0 = make_float2(wb.x, wb.y), b1 = make_float2(wb.z, wb.w);
            re0 = __ffma2_rn(wa[m], b0, re0);
            im0 = __ffma2_rn(wc[m], b0, im0);
            re1 = __ffma2_rn(wa[m + 1], b1, re1);
            im1 = __ffma2_rn(wc[m + 1], b1, im1);
        }
        const float re = (hsum(re0) + hsum(re1)) * inv_tr;
        const float im = (hsum(im0) + hsum(im1)) * inv_tr;
        const bool upper = arow < b;
        packed[arow * PK + b] = upper ? re : im;
        packed[b * PK + arow] = upper ? -im : re;
    }
    if (active && j == 0) a.trace_out[c] = (double)tr_hi + (double)tr_lo;
    __syncwarp();

    // ---- 5. store packed rho (FP32) and its exact bf16 split ----------------------------------
    if (active) {
        float *dst = a.rho_out + c * a.d_pad;
        for (int e = 4 * j; e < d; e += 4 * D) {
            // entries e .. e+3 of the row-major packed rho, staged with row stride PK
            auto staged = [&](int ee) { return packed[(ee / D) * PK + (ee % D)]; };
            const float4 v = make_float4(staged(e), staged(e + 1), staged(e + 2), staged(e + 3));
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
            if (a.split_tf) {   // TF32 hi = v rounded to 11 significant bits, lo = TF32(v - hi)
                const float4 hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
                float *sp = a.split_tf + c * (int64_t)a.tf_splits * a.d_pad + e;
                *reinterpret_cast<float4 *>(sp) = hi;
                if (a.tf_splits == 2)
                    *reinterpret_cast<float4 *>(sp + a.d_pad) = make_float4(
                        tf32_rna(v.x - hi.x), tf32_rna(v.y - hi.y), tf32_rna(v.z - hi.z), tf32_rna(v.w - hi.w));
            }
        }
    }
}

// ---- five qubits (D = 32): one warp per chain ----------------------------------------------
// The same algorithm with the same lane ownership (lane j: column j, then row j), but at D = 32 a
// lane cannot also hold the operand it is multiplied with, so that operand is streamed from
// shared memory four complex entries (two 128-bit loads) at a time.  With PASSES = 3 the
// refinement of U runs as in the D <= 16 kernel (refine_pass); its copy of H and the packed R take
// 4.2 KB more per chain, so that form runs two chains per CTA (THREADS = 64): five CTAs, ten
// warps, on an SM.
template <int PASSES = 2, int THREADS = kThreads>
struct WideShape {
    static constexpr int D = 32;
    static constexpr int d = D * D;
    static constexpr int chains_per_block = THREADS / D;
    static constexpr int qcol = D + 4;                      // floats per column of a Q plane
    static constexpr int pk_stride = D + 1;
    static constexpr int area_a = 2 * D * qcol;             // Q planes, then W as two planes of stride qcol
    static constexpr int area_b = 2 * D * D;                // F planes (PASSES = 3: H's columns), then the staged rho
    static constexpr int area_r = (PASSES == 3) ? D * (D + 1) : 0;   // PASSES = 3: packed R
    static constexpr int smem_floats = (area_a + area_b + area_r + 31) / 32 * 32 + 16;
};
using Wide = WideShape<>;
static_assert(Wide::area_b >= Wide::D * Wide::pk_stride, "areas");

template <int PASSES, int THREADS = kThreads>
__global__ void __launch_bounds__(THREADS, 3 * kThreads / THREADS) propose_kernel_d32(ProposeArgs a) {
    using S = WideShape<PASSES, THREADS>;
    constexpr int D = S::D, d = S::d, nx = 4 * d, QC = S::qcol, PK = S::pk_stride;
    extern __shared__ __align__(16) float smem[];
    const int j = threadIdx.x % D;
    const int g = threadIdx.x / D;
    const int64_t c = (int64_t)blockIdx.x * S::chains_per_block + g;
    const bool active = c < a.rows;
    const uint32_t step = (a.step_dev && a.mode == MODE_STEP) ? a.step_dev->step : a.step;
    float *sm = smem + g * S::smem_floats;
    float *qre = sm, *qim = sm + D * QC;                 // Q planes (column stride QC)
    float *wre = sm, *wim = sm + D * QC;                 // W planes (row stride QC), replace Q
    float *fre = sm + S::area_a, *fim = fre + D * D;     // F column-major (stride D), re / im planes
    float *packed = sm + S::area_a;                      // staged rho (row stride PK), replaces F
    float *hre = sm + S::area_a, *him = hre + D * D;     // PASSES = 3: H's columns (stride D), in area B
    float2 *rpk = reinterpret_cast<float2 *>(sm + S::area_a + S::area_b);   // PASSES = 3: packed R

    // ---- 1. latent proposal (as in the D <= 16 kernel: lane j owns column j of each part) ------
    float coef_y = 1.0f, coef_eta = 0.0f;
    int cur = 0;
    if (active && a.mode == MODE_STEP) {
        cur = a.cur[c];
        const float2 cf = a.coef[c];
        coef_y = cf.x;
        coef_eta = cf.y;
    } else if (a.mode == MODE_INIT) {
        coef_y = 0.0f;
        coef_eta = 1.0f;
    }
    const int64_t cc = active ? c : 0;
    const uint32_t chain_id = (uint32_t)(a.chain_offset + cc);
    const uint32_t tag = (a.mode == MODE_INIT) ? TAG_INIT : TAG_PROPOSAL;
    const float *ysrc = a.y + ((int64_t)cur * a.R + cc) * nx;
    float *ydst = a.y + ((int64_t)(1 - cur) * a.R + cc) * nx;
    const float *gsrc = (a.mode == MODE_EVAL) ? a.x_eval + cc * nx : ydst;
    float2 hr[D / 2], hi[D / 2];   // H's column j, entries (2p, 2p + 1) in pair p
#pragma unroll 1
    for (int part = 0; part < 4; ++part) {
        const int e0 = part * d + j * D;
#pragma unroll
        for (int q = 0; q < D / 4; ++q) {
            float4 y0 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (active && a.mode == MODE_STEP) y0 = *reinterpret_cast<const float4 *>(ysrc + e0 + 4 * q);
            if (active && a.mode == MODE_EVAL) y0 = *reinterpret_cast<const float4 *>(a.x_eval + cc * nx + e0 + 4 * q);
            float4 yn = y0;
            if (a.mode != MODE_EVAL) {
                const uint4 w = Philox::block(make_uint4((uint32_t)(e0 / 4 + q), step, chain_id, tag), a.rk);
                float z0, z1, z2, z3;
                gaussian_pair_fast(w.x, w.y, z0, z1);
                gaussian_pair_fast(w.z, w.w, z2, z3);
                yn.x = __fmaf_rn(coef_y, y0.x, coef_eta * z0);
                yn.y = __fmaf_rn(coef_y, y0.y, coef_eta * z1);
                yn.z = __fmaf_rn(coef_y, y0.z, coef_eta * z2);
                yn.w = __fmaf_rn(coef_y, y0.w, coef_eta * z3);
                if (active) *reinterpret_cast<float4 *>(ydst + e0 + 4 * q) = yn;
            }
            if (part == 2) {
                hr[2 * q] = make_float2(yn.x, yn.y);
                hr[2 * q + 1] = make_float2(yn.z, yn.w);
            } else if (part == 3) {
                hi[2 * q] = make_float2(yn.x, yn.y);
                hi[2 * q + 1] = make_float2(yn.z, yn.w);
            }
        }
    }
    if constexpr (PASSES == 3) {   // H's original columns, for the refinement after the sweep
        store_column2<D>(hre + j * D, hr);
        store_column2<D>(him + j * D, hi);
    }

    // ---- 2a. modified Gram-Schmidt, the published column streamed in chunks --------------------
    // As in the D <= 16 kernel: every lane forms r = v_k^dag h (lane k's is |v_k|^2, shuffled to
    // the others), one uniform rsqrt, a branch-free projection (zero coefficient on lanes
    // j <= k), and the lanes j < k form the Gram entries of the re-orthogonalisation.
    float inv_own = 0.0f;
#pragma unroll 1
    for (int k = 0; k < (PASSES > 0 ? D : 0); ++k) {   // (PASSES = 0, the Hilbert-Schmidt prior: no QR)
        if (j == k) {
            store_column2<D>(qre + k * QC, hr);
            store_column2<D>(qim + k * QC, hi);
        }
        __syncwarp();
        const float *vre = qre + k * QC, *vim = qim + k * QC;
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0, b0 = a0, b1 = a0, b2 = a0, b3 = a0;
#pragma unroll
        for (int p = 0; p < D / 2; p += 2) {
            const float4 vr4 = *reinterpret_cast<const float4 *>(vre + 2 * p);
            const float4 vi4 = *reinterpret_cast<const float4 *>(vim + 2 * p);
            const float2 vr0 = make_float2(vr4.x, vr4.y), vr1 = make_float2(vr4.z, vr4.w);
            const float2 vi0 = make_float2(vi4.x, vi4.y), vi1 = make_float2(vi4.z, vi4.w);
            a0 = __ffma2_rn(vr0, hr[p], a0);
            a1 = __ffma2_rn(vi0, hi[p], a1);
            b0 = __ffma2_rn(vr0, hi[p], b0);
            b1 = __ffma2_rn(vi0, hr[p], b1);
            a2 = __ffma2_rn(vr1, hr[p + 1], a2);
            a3 = __ffma2_rn(vi1, hi[p + 1], a3);
            b2 = __ffma2_rn(vr1, hi[p + 1], b2);
            b3 = __ffma2_rn(vi1, hr[p + 1], b3);
        }
        const float rr = (hsum(a0) + hsum(a1)) + (hsum(a2) + hsum(a3));
        const float ri = (hsum(b0) - hsum(b1)) + (hsum(b2) - hsum(b3));
        const float nk = __shfl_sync(0xffffffffu, rr, k);   // |v_k|^2 from lane k
        const float rs = rsqrtf(nk);
        const float coef = (j > k) ? rs * rs : 0.0f;
        const float sr = rr * coef, si = ri * coef;
        const float2 msr = make_float2(-sr, -sr), psi = make_float2(si, si), msi = make_float2(-si, -si);
#pragma unroll
        for (int p = 0; p < D / 2; p += 2) {
            const float4 vr4 = *reinterpret_cast<const float4 *>(vre + 2 * p);
            const float4 vi4 = *reinterpret_cast<const float4 *>(vim + 2 * p);
            const float2 vr0 = make_float2(vr4.x, vr4.y), vr1 = make_float2(vr4.z, vr4.w);
            const float2 vi0 = make_float2(vi4.x, vi4.y), vi1 = make_float2(vi4.z, vi4.w);
            hr[p] = __ffma2_rn(msr, vr0, __ffma2_rn(psi, vi0, hr[p]));
            hi[p] = __ffma2_rn(msr, vi0, __ffma2_rn(msi, vr0, hi[p]));
            hr[p + 1] = __ffma2_rn(msr, vr1, __ffma2_rn(psi, vi1, hr[p + 1]));
            hi[p + 1] = __ffma2_rn(msr, vi1, __ffma2_rn(msi, vr1, hi[p + 1]));
        }
        inv_own = (j == k) ? rs : inv_own;
        if constexpr (PASSES == 2) {
            if (j < k) {
                const float sc = inv_own * rs;   // E_jk = conj(r) / (|v_j| |v_k|), j < k
                fre[k * D + j] = rr * sc;
                fim[k * D + j] = -ri * sc;
            }
        }
        if constexpr (PASSES == 3) {   // R for the refinement's solve, as in the D <= 16 kernel
            if (j > k) rpk[j * (j + 1) / 2 + k] = make_float2(rr * rs, ri * rs);
            if (j == k) rpk[k * (k + 1) / 2 + k] = make_float2(nk * rs, rs);
        }
    }
    if constexpr (PASSES > 0) {   // normalise the own column and publish it
        const float2 sc = make_float2(inv_own, inv_own);
#pragma unroll
        for (int p = 0; p < D / 2; ++p) {
            hr[p] = __fmul2_rn(hr[p], sc);
            hi[p] = __fmul2_rn(hi[p], sc);
        }
        __syncwarp();
        store_column2<D>(qre + j * QC, hr);
        store_column2<D>(qim + j * QC, hi);
        __syncwarp();
    }

    if constexpr (PASSES == 3) {
        // ---- 2b. refinement of Q1 to the QR factor of H beyond FP32 (the D <= 16 kernel's step 2b:
        // error-free M and N rows per lane, the triangular solve, U = Q1 - Q1 Y^dag, repeated while
        // the chain's largest |Y| entry exceeds kRefineTol) ----------------------------------------
        const float ymax = refine_pass<D, QC>(hr, hi, qre, qim, hre, him, rpk, gsrc, j, false, true);
        if (__any_sync(0xffffffffu, ymax > kRefineTol)) refine_more<D, QC>(qre, qim, hre, him, rpk, gsrc, j, ymax);
    }

    if constexpr (PASSES == 2) {
        // ---- 2b. Q2 = Q1 (I - F): F's diagonal, then row a of Q1 (I - F) (as in D <= 16) ----------
        {
            float2 n = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < D / 2; ++p) n = __ffma2_rn(hr[p], hr[p], __ffma2_rn(hi[p], hi[p], n));
            fre[j * D + j] = 0.5f * (hsum(n) - 1.0f);
            fim[j * D + j] = 0.0f;
            if (j + 1 < D) {
                fre[j * D + j + 1] = 0.0f;
                fim[j * D + j + 1] = 0.0f;
            }
        }
        __syncwarp();
        {
            float2 xr[D / 2], xi[D / 2];
#pragma unroll
            for (int p = 0; p < D / 2; ++p) {
                xr[p] = make_float2(qre[(2 * p) * QC + j], qre[(2 * p + 1) * QC + j]);
                xi[p] = make_float2(qim[(2 * p) * QC + j], qim[(2 * p + 1) * QC + j]);
            }
#pragma unroll
            for (int m = D - 1; m >= 0; --m) {
                float2 ca = make_float2(0.f, 0.f), cb = ca, cc2 = ca, cd = ca;
#pragma unroll
                for (int p = 0; 2 * p <= m; ++p) {
                    float2 fx, fy;   // F[2p][m], F[2p+1][m]
                    if ((p & 1) == 0) {
                        const float4 f4x = *reinterpret_cast<const float4 *>(fre + m * D + 2 * p);
                        const float4 f4y = *reinterpret_cast<const float4 *>(fim + m * D + 2 * p);
                        fx = make_float2(f4x.x, f4x.y);
                        fy = make_float2(f4y.x, f4y.y);
                    } else {
                        fx = *reinterpret_cast<const float2 *>(fre + m * D + 2 * p);
                        fy = *reinterpret_cast<const float2 *>(fim + m * D + 2 * p);
                    }
                    ca = __ffma2_rn(xr[p], fx, ca);
                    cb = __ffma2_rn(xi[p], fy, cb);
                    cc2 = __ffma2_rn(xr[p], fy, cc2);
                    cd = __ffma2_rn(xi[p], fx, cd);
                }
                const float dr = hsum(ca) - hsum(cb), di = hsum(cc2) + hsum(cd);
                if (m & 1) {
                    xr[m / 2].y -= dr;
                    xi[m / 2].y -= di;
                } else {
                    xr[m / 2].x -= dr;
                    xi[m / 2].x -= di;
                }
            }
#pragma unroll
            for (int p = 0; p < D / 2; ++p) {
                qre[(2 * p) * QC + j] = xr[p].x;
                qre[(2 * p + 1) * QC + j] = xr[p].y;
                qim[(2 * p) * QC + j] = xi[p].x;
                qim[(2 * p + 1) * QC + j] = xi[p].y;
            }
        }
        __syncwarp();
    }

    // ---- 3. W[:, j] = G[:, j] + sum_k U[:, k] G[k, j]: pairs of rows, U streamed, G[k, j] broadcast
    float2 wr[D / 2], wi[D / 2];
#pragma unroll
    for (int p = 0; p < D / 2; ++p) wr[p] = wi[p] = make_float2(0.f, 0.f);
    // G[k0..k0+3, j] from y' (L2), requested one group ahead of its use
    float4 g4r_next = make_float4(0.f, 0.f, 0.f, 0.f), g4i_next = g4r_next;
    if (active && PASSES > 0) {
        g4r_next = *reinterpret_cast<const float4 *>(gsrc + j * D);
        g4i_next = *reinterpret_cast<const float4 *>(gsrc + d + j * D);
    }
#pragma unroll 1
    for (int k0 = 0; k0 < (PASSES > 0 ? D : 0); k0 += 4) {
        const float4 g4r = g4r_next, g4i = g4i_next;
        if (active && k0 + 4 < D) {
            g4r_next = *reinterpret_cast<const float4 *>(gsrc + j * D + k0 + 4);
            g4i_next = *reinterpret_cast<const float4 *>(gsrc + d + j * D + k0 + 4);
        }
        const float gkr[4] = {g4r.x, g4r.y, g4r.z, g4r.w}, gki[4] = {g4i.x, g4i.y, g4i.z, g4i.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float *ure = qre + (k0 + u) * QC, *uim = qim + (k0 + u) * QC;
            const float2 pgr = make_float2(gkr[u], gkr[u]), pgi = make_float2(gki[u], gki[u]);
            const float2 mgi = make_float2(-gki[u], -gki[u]);
#pragma unroll
            for (int p = 0; p < D / 2; p += 2) {
                const float4 ur = *reinterpret_cast<const float4 *>(ure + 2 * p);
                const float4 ui = *reinterpret_cast<const float4 *>(uim + 2 * p);
                const float2 ur0 = make_float2(ur.x, ur.y), ur1 = make_float2(ur.z, ur.w);
                const float2 ui0 = make_float2(ui.x, ui.y), ui1 = make_float2(ui.z, ui.w);
                wr[p] = __ffma2_rn(ur0, pgr, __ffma2_rn(ui0, mgi, wr[p]));
                wi[p] = __ffma2_rn(ur0, pgi, __ffma2_rn(ui0, pgr, wi[p]));
                wr[p + 1] = __ffma2_rn(ur1, pgr, __ffma2_rn(ui1, mgi, wr[p + 1]));
                wi[p + 1] = __ffma2_rn(ur1, pgi, __ffma2_rn(ui1, pgr, wi[p + 1]));
            }
        }
    }
    if (active) {   // + G[:, j]
#pragma unroll
        for (int p = 0; p < D / 2; p += 2) {
            const float4 gr4 = *reinterpret_cast<const float4 *>(gsrc + j * D + 2 * p);
            const float4 gi4 = *reinterpret_cast<const float4 *>(gsrc + d + j * D + 2 * p);
            wr[p] = __fadd2_rn(wr[p], make_float2(gr4.x, gr4.y));
            wr[p + 1] = __fadd2_rn(wr[p + 1], make_float2(gr4.z, gr4.w));
            wi[p] = __fadd2_rn(wi[p], make_float2(gi4.x, gi4.y));
            wi[p + 1] = __fadd2_rn(wi[p + 1], make_float2(gi4.z, gi4.w));
        }
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < D / 2; ++p) {   // W row-major, real and imaginary planes (replace Q)
        wre[(2 * p) * QC + j] = wr[p].x;
        wre[(2 * p + 1) * QC + j] = wr[p].y;
        wim[(2 * p) * QC + j] = wi[p].x;
        wim[(2 * p + 1) * QC + j] = wi[p].y;
    }
    __syncwarp();

    // ---- 4. rho = W W^dag / Tr, lane a: entries (a, a + t mod D), row b streamed --------------
    // Re (W W^dag)_ab = sum Re W_am Re W_bm + Im W_am Im W_bm and Im = sum Im W_am Re W_bm -
    // Re W_am Im W_bm, on pairs of columns m.  For t = D/2 lanes a and a + D/2 both form the pair
    // {a, a + D/2}; the results are bitwise equal (the same products in the same order), so both
    // stores may stand.
    const int arow = j;
    float2 war[D / 2], wai[D / 2];
#pragma unroll
    for (int p = 0; p < D / 2; p += 2) {
        const float4 r4 = *reinterpret_cast<const float4 *>(wre + arow * QC + 2 * p);
        const float4 i4 = *reinterpret_cast<const float4 *>(wim + arow * QC + 2 * p);
        war[p] = make_float2(r4.x, r4.y);
        war[p + 1] = make_float2(r4.z, r4.w);
        wai[p] = make_float2(i4.x, i4.y);
        wai[p + 1] = make_float2(i4.z, i4.w);
    }
    float diag;
    {
        float2 d0 = make_float2(0.f, 0.f), d1 = d0;
#pragma unroll
        for (int p = 0; p < D / 2; ++p) {
            d0 = __ffma2_rn(war[p], war[p], d0);
            d1 = __ffma2_rn(wai[p], wai[p], d1);
        }
        diag = hsum(d0) + hsum(d1);
    }
    const float inv_tr = 1.0f / group_sum<D>(diag);
    const float diag_n = diag * inv_tr;
    float tr_hi, tr_lo;
    group_sum_exact<D>(diag_n, tr_hi, tr_lo);
    __syncwarp();   // every lane holds its W row before F's area becomes the staged rho
    packed[arow * PK + arow] = diag_n;
#pragma unroll 1
    for (int t = 1; t <= D / 2; ++t) {
        const int b = (arow + t) & (D - 1);
        float2 re = make_float2(0.f, 0.f), ima = re, imb = re;
#pragma unroll
        for (int p = 0; p < D / 2; p += 2) {
            const float4 r4 = *reinterpret_cast<const float4 *>(wre + b * QC + 2 * p);
            const float4 i4 = *reinterpret_cast<const float4 *>(wim + b * QC + 2 * p);
            const float2 br0 = make_float2(r4.x, r4.y), br1 = make_float2(r4.z, r4.w);
            const float2 bi0 = make_float2(i4.x, i4.y), bi1 = make_float2(i4.z, i4.w);
            re = __ffma2_rn(wai[p], bi0, __ffma2_rn(war[p], br0, re));
            ima = __ffma2_rn(wai[p], br0, ima);
            imb = __ffma2_rn(war[p], bi0, imb);
            re = __ffma2_rn(wai[p + 1], bi1, __ffma2_rn(war[p + 1], br1, re));
            ima = __ffma2_rn(wai[p + 1], br1, ima);
            imb = __ffma2_rn(war[p + 1], bi1, imb);
        }
        const float rv = hsum(re) * inv_tr;
        const float iv = (hsum(ima) - hsum(imb)) * inv_tr;
        const bool upper = arow < b;
        packed[arow * PK + b] = upper ? rv : iv;
        packed[b * PK + arow] = upper ? -iv : rv;
    }
    if (active && j == 0) a.trace_out[c] = (double)tr_hi + (double)tr_lo;
    __syncwarp();

    // ---- 5. store packed rho (FP32) and its exact bf16 split ----------------------------------
    if (active) {
        float *dst = a.rho_out + c * a.d_pad;
        for (int e = 4 * j; e < d; e += 4 * D) {
            auto staged = [&](int ee) { return packed[(ee / D) * PK + (ee % D)]; };
            const float4 v = make_float4(staged(e), staged(e + 1), staged(e + 2), staged(e + 3));
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

// ---------------------------------------------------------------------------------------
// D = 64 (six qubits): one 128-thread CTA per chain, two threads per column (thread 2 j + h holds
// rows 32 h .. 32 h + 31 of column j).  The same steps as the kernels above, with CTA barriers
// where those use warp ones: the latent proposal and H's column half in registers; modified
// Gram-Schmidt with each column normalised by its owner pair and published to shared memory
// (the others project it out; pairs whose column is final form the Gram entries); the
// first-order re-orthogonalisation Q1 (I - F) (R21) by rows; W = (U + I) G by column halves;
// the Hermitian half of W W^dag by rows, the two threads of a row splitting its columns.
// ---------------------------------------------------------------------------------------
struct Wide64 {
    static constexpr int D = 64;
    static constexpr int d = D * D;
    static constexpr int threads = 128;
    // floats per column of a Q plane (per row of W): entry i sits at i + 4 (i / 32), so the two
    // halves a thread pair works on fall in different 16-byte bank groups and the eight float4
    // accesses of a quarter warp in distinct ones (72 = 18 groups of 4 floats per column)
    static constexpr int qcol = D + 8;
    static constexpr int pk_stride = D + 1;
    static constexpr int area_a = 2 * D * qcol;         // Q planes, then W as two planes of row stride qcol
    static constexpr int area_b = 2 * D * D;            // F planes (column-major), then the staged rho
    static constexpr int smem_floats = area_a + area_b + 2 * D + 32;
};
static_assert(Wide64::area_b >= Wide64::D * Wide64::pk_stride, "areas");

template <int PASSES>
__global__ void __launch_bounds__(Wide64::threads, 3) propose_kernel_d64(ProposeArgs a) {
    using S = Wide64;
    constexpr int D = S::D, d = S::d, nx = 4 * d, QC = S::qcol, PK = S::pk_stride, H2 = D / 2;
    extern __shared__ __align__(16) float smem[];
    float *qre = smem, *qim = smem + D * QC;             // Q planes (column stride QC)
    float *wre = smem, *wim = smem + D * QC;             // W planes (row stride QC), replace Q
    float *fre = smem + S::area_a, *fim = fre + D * D;   // F column-major (F[p][m] at m D + p)
    float *packed = smem + S::area_a;                    // staged rho (row stride PK), replaces F
    float *rowv = smem + S::area_a + S::area_b;          // [D] per-row values (diagonal of W W^dag)
    const int t = threadIdx.x;
    const int j = t >> 1, hh = t & 1, r0 = H2 * hh;      // column (or row) j, half hh
    const int r0s = r0 + 4 * hh;                         // where half hh starts within a column (row)
    const int js = j + 4 * (j >> 5);                     // where entry j sits within a column (row)
    const unsigned pair_mask = 3u << ((t & 31) & ~1);
    const int64_t c = blockIdx.x;                        // one chain per CTA; the grid is exactly rows
    const uint32_t step = (a.step_dev && a.mode == MODE_STEP) ? a.step_dev->step : a.step;

    // ---- 1. latent proposal: this thread's 32 entries of column j of each part -----------------
    float coef_y = 1.0f, coef_eta = 0.0f;
    int cur = 0;
    if (a.mode == MODE_STEP) {
        cur = a.cur[c];
        const float2 cf = a.coef[c];
        coef_y = cf.x;
        coef_eta = cf.y;
    } else if (a.mode == MODE_INIT) {
        coef_y = 0.0f;
        coef_eta = 1.0f;
    }
    const uint32_t chain_id = (uint32_t)(a.chain_offset + c);
    const uint32_t tag = (a.mode == MODE_INIT) ? TAG_INIT : TAG_PROPOSAL;
    const float *ysrc = a.y + ((int64_t)cur * a.R + c) * nx;
    float *ydst = a.y + ((int64_t)(1 - cur) * a.R + c) * nx;
    const float *gsrc = (a.mode == MODE_EVAL) ? a.x_eval + c * nx : ydst;
    float2 hr[H2 / 2], hi[H2 / 2];   // rows r0 + 2p, r0 + 2p + 1 of H's column j in pair p
#pragma unroll 1
    for (int part = 0; part < 4; ++part) {
        const int e0 = part * d + j * D + r0;
#pragma unroll
        for (int q = 0; q < H2 / 4; ++q) {
            float4 y0 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a.mode == MODE_STEP) y0 = *reinterpret_cast<const float4 *>(ysrc + e0 + 4 * q);
            if (a.mode == MODE_EVAL) y0 = *reinterpret_cast<const float4 *>(a.x_eval + c * nx + e0 + 4 * q);
            float4 yn = y0;
            if (a.mode != MODE_EVAL) {
                const uint4 w = Philox::block(make_uint4((uint32_t)(e0 / 4 + q), step, chain_id, tag), a.rk);
                float z0, z1, z2, z3;
                gaussian_pair_fast(w.x, w.y, z0, z1);
                gaussian_pair_fast(w.z, w.w, z2, z3);
                yn.x = __fmaf_rn(coef_y, y0.x, coef_eta * z0);
                yn.y = __fmaf_rn(coef_y, y0.y, coef_eta * z1);
                yn.z = __fmaf_rn(coef_y, y0.z, coef_eta * z2);
                yn.w = __fmaf_rn(coef_y, y0.w, coef_eta * z3);
                *reinterpret_cast<float4 *>(ydst + e0 + 4 * q) = yn;
            }
            if (part == 2) {
                hr[2 * q] = make_float2(yn.x, yn.y);
                hr[2 * q + 1] = make_float2(yn.z, yn.w);
            } else if (part == 3) {
                hi[2 * q] = make_float2(yn.x, yn.y);
                hi[2 * q + 1] = make_float2(yn.z, yn.w);
            }
        }
    }
    __syncthreads();   // y' (read back as G) is written

    // ---- 2a. modified Gram-Schmidt: q_k = v_k / |v_k| published by its pair, projected out ------
#pragma unroll 1
    for (int k = 0; k < (PASSES > 0 ? D : 0); ++k) {   // (PASSES = 0, the Hilbert-Schmidt prior: no QR)
        if (j == k) {
            float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < H2 / 2; ++p) n2 = __ffma2_rn(hr[p], hr[p], __ffma2_rn(hi[p], hi[p], n2));
            float n = hsum(n2);
            n += __shfl_xor_sync(pair_mask, n, 1);
            const float2 rs = make_float2(rsqrtf(n), rsqrtf(n));
#pragma unroll
            for (int p = 0; p < H2 / 2; ++p) {
                hr[p] = __fmul2_rn(hr[p], rs);
                hi[p] = __fmul2_rn(hi[p], rs);
            }
            store_column2<H2>(qre + k * QC + r0s, hr);
            store_column2<H2>(qim + k * QC + r0s, hi);
        }
        __syncthreads();
        // r = q_k^dag h over this half, then both halves
        const float *vre = qre + k * QC + r0s, *vim = qim + k * QC + r0s;
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
        for (int p = 0; p < H2 / 2; p += 2) {
            const float4 vr4 = *reinterpret_cast<const float4 *>(vre + 2 * p);
            const float4 vi4 = *reinterpret_cast<const float4 *>(vim + 2 * p);
            const float2 vr0 = make_float2(vr4.x, vr4.y), vr1 = make_float2(vr4.z, vr4.w);
            const float2 vi0 = make_float2(vi4.x, vi4.y), vi1 = make_float2(vi4.z, vi4.w);
            a0 = __ffma2_rn(vr0, hr[p], __ffma2_rn(vr1, hr[p + 1], a0));
            a1 = __ffma2_rn(vi0, hi[p], __ffma2_rn(vi1, hi[p + 1], a1));
            b0 = __ffma2_rn(vr0, hi[p], __ffma2_rn(vr1, hi[p + 1], b0));
            b1 = __ffma2_rn(vi0, hr[p], __ffma2_rn(vi1, hr[p + 1], b1));
        }
        float rr = hsum(a0) + hsum(a1), ri = hsum(b0) - hsum(b1);
        rr += __shfl_xor_sync(0xffffffffu, rr, 1);
        ri += __shfl_xor_sync(0xffffffffu, ri, 1);
        if (j > k) {   // h -= r q_k
            const float2 msr = make_float2(-rr, -rr), psi = make_float2(ri, ri), msi = make_float2(-ri, -ri);
#pragma unroll
            for (int p = 0; p < H2 / 2; p += 2) {
                const float4 vr4 = *reinterpret_cast<const float4 *>(vre + 2 * p);
                const float4 vi4 = *reinterpret_cast<const float4 *>(vim + 2 * p);
                const float2 vr0 = make_float2(vr4.x, vr4.y), vr1 = make_float2(vr4.z, vr4.w);
                const float2 vi0 = make_float2(vi4.x, vi4.y), vi1 = make_float2(vi4.z, vi4.w);
                hr[p] = __ffma2_rn(msr, vr0, __ffma2_rn(psi, vi0, hr[p]));
                hi[p] = __ffma2_rn(msr, vi0, __ffma2_rn(msi, vr0, hi[p]));
                hr[p + 1] = __ffma2_rn(msr, vr1, __ffma2_rn(psi, vi1, hr[p + 1]));
                hi[p + 1] = __ffma2_rn(msr, vi1, __ffma2_rn(msi, vr1, hi[p + 1]));
            }
        } else if (PASSES == 2 && j < k && hh == 0) {   // E_jk = q_j^dag q_k = conj(q_k^dag q_j)
            fre[k * D + j] = rr;
            fim[k * D + j] = -ri;
        }
    }

    if constexpr (PASSES == 2) {
        {   // F's diagonal: (|q_j|^2 - 1) / 2
            float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < H2 / 2; ++p) n2 = __ffma2_rn(hr[p], hr[p], __ffma2_rn(hi[p], hi[p], n2));
            float n = hsum(n2);
            n += __shfl_xor_sync(0xffffffffu, n, 1);
            if (hh == 0) {
                fre[j * D + j] = 0.5f * (n - 1.0f);
                fim[j * D + j] = 0.0f;
            }
        }
        __syncthreads();
        // ---- 2b. Q2 = Q1 (I - F): row a = j, the columns m of parity hh ------------------------
        float2 q2[H2];   // (re, im) of Q2[a][2 mm + hh]
#pragma unroll 1
        for (int mm = 0; mm < H2; ++mm) {
            const int m = 2 * mm + hh;
            float2 acc = make_float2(0.f, 0.f), acc2 = acc;   // sum_p Q1[a][p] F[p][m] as (re, im) pairs
            for (int p = 0; p <= m; ++p) {
                const float xr = qre[p * QC + js], xi = qim[p * QC + js];
                const float fr = fre[m * D + p], fi = fim[m * D + p];
                acc = __ffma2_rn(make_float2(xr, xr), make_float2(fr, fi), acc);     // (xr fr, xr fi)
                acc2 = __ffma2_rn(make_float2(xi, xi), make_float2(fi, fr), acc2);   // (xi fi, xi fr)
            }
            q2[mm] = make_float2(qre[m * QC + js] - (acc.x - acc2.x), qim[m * QC + js] - (acc.y + acc2.y));
        }
        __syncthreads();
#pragma unroll
        for (int mm = 0; mm < H2; ++mm) {
            qre[(2 * mm + hh) * QC + js] = q2[mm].x;
            qim[(2 * mm + hh) * QC + js] = q2[mm].y;
        }
        __syncthreads();
    } else {
        __syncthreads();
    }

    // ---- 3. W[:, j] = G[:, j] + sum_k U[:, k] G[k, j] over this half's rows --------------------
    float2 wr[H2 / 2], wi[H2 / 2];
#pragma unroll
    for (int p = 0; p < H2 / 2; ++p) wr[p] = wi[p] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int k0 = 0; k0 < (PASSES > 0 ? D : 0); k0 += 4) {
        const float4 g4r = *reinterpret_cast<const float4 *>(gsrc + j * D + k0);
        const float4 g4i = *reinterpret_cast<const float4 *>(gsrc + d + j * D + k0);
        const float gkr[4] = {g4r.x, g4r.y, g4r.z, g4r.w}, gki[4] = {g4i.x, g4i.y, g4i.z, g4i.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float *ure = qre + (k0 + u) * QC + r0s, *uim = qim + (k0 + u) * QC + r0s;
            const float2 pgr = make_float2(gkr[u], gkr[u]), pgi = make_float2(gki[u], gki[u]);
            const float2 mgi = make_float2(-gki[u], -gki[u]);
#pragma unroll
            for (int p = 0; p < H2 / 2; p += 2) {
                const float4 ur = *reinterpret_cast<const float4 *>(ure + 2 * p);
                const float4 ui = *reinterpret_cast<const float4 *>(uim + 2 * p);
                const float2 ur0 = make_float2(ur.x, ur.y), ur1 = make_float2(ur.z, ur.w);
                const float2 ui0 = make_float2(ui.x, ui.y), ui1 = make_float2(ui.z, ui.w);
                wr[p] = __ffma2_rn(ur0, pgr, __ffma2_rn(ui0, mgi, wr[p]));
                wi[p] = __ffma2_rn(ur0, pgi, __ffma2_rn(ui0, pgr, wi[p]));
                wr[p + 1] = __ffma2_rn(ur1, pgr, __ffma2_rn(ui1, mgi, wr[p + 1]));
                wi[p + 1] = __ffma2_rn(ur1, pgi, __ffma2_rn(ui1, pgr, wi[p + 1]));
            }
        }
    }
#pragma unroll
    for (int p = 0; p < H2 / 2; p += 2) {   // + G[:, j]
        const float4 gr4 = *reinterpret_cast<const float4 *>(gsrc + j * D + r0 + 2 * p);
        const float4 gi4 = *reinterpret_cast<const float4 *>(gsrc + d + j * D + r0 + 2 * p);
        wr[p] = __fadd2_rn(wr[p], make_float2(gr4.x, gr4.y));
        wr[p + 1] = __fadd2_rn(wr[p + 1], make_float2(gr4.z, gr4.w));
        wi[p] = __fadd2_rn(wi[p], make_float2(gi4.x, gi4.y));
        wi[p + 1] = __fadd2_rn(wi[p + 1], make_float2(gi4.z, gi4.w));
    }
    __syncthreads();   // U is read by every thread before W replaces it
#pragma unroll
    for (int p = 0; p < H2 / 2; ++p) {   // W row-major, real and imaginary planes
        wre[(r0 + 2 * p) * QC + js] = wr[p].x;
        wre[(r0 + 2 * p + 1) * QC + js] = wr[p].y;
        wim[(r0 + 2 * p) * QC + js] = wi[p].x;
        wim[(r0 + 2 * p + 1) * QC + js] = wi[p].y;
    }
    __syncthreads();

    // ---- 4. rho = W W^dag / Tr: row a = j, this thread's half of the columns m ------------------
    const int arow = j;
    float2 war[H2 / 2], wai[H2 / 2];
#pragma unroll
    for (int p = 0; p < H2 / 2; p += 2) {
        const float4 r4 = *reinterpret_cast<const float4 *>(wre + arow * QC + r0s + 2 * p);
        const float4 i4 = *reinterpret_cast<const float4 *>(wim + arow * QC + r0s + 2 * p);
        war[p] = make_float2(r4.x, r4.y);
        war[p + 1] = make_float2(r4.z, r4.w);
        wai[p] = make_float2(i4.x, i4.y);
        wai[p + 1] = make_float2(i4.z, i4.w);
    }
    {
        float2 d0 = make_float2(0.f, 0.f), d1 = d0;
#pragma unroll
        for (int p = 0; p < H2 / 2; ++p) {
            d0 = __ffma2_rn(war[p], war[p], d0);
            d1 = __ffma2_rn(wai[p], wai[p], d1);
        }
        float diag = hsum(d0) + hsum(d1);
        diag += __shfl_xor_sync(0xffffffffu, diag, 1);
        if (hh == 0) rowv[arow] = diag;
    }
    __syncthreads();
    float tr = 0.0f;   // Tr W W^dag in row order (every thread alike)
    for (int r = 0; r < D; ++r) tr += rowv[r];
    const float inv_tr = 1.0f / tr;
    if (hh == 0) packed[arow * PK + arow] = rowv[arow] * inv_tr;
#pragma unroll 1
    for (int s = 1; s <= D / 2; ++s) {
        const int b = (arow + s) & (D - 1);
        float2 re = make_float2(0.f, 0.f), ima = re, imb = re;
#pragma unroll
        for (int p = 0; p < H2 / 2; p += 2) {
            const float4 r4 = *reinterpret_cast<const float4 *>(wre + b * QC + r0s + 2 * p);
            const float4 i4 = *reinterpret_cast<const float4 *>(wim + b * QC + r0s + 2 * p);
            const float2 br0 = make_float2(r4.x, r4.y), br1 = make_float2(r4.z, r4.w);
            const float2 bi0 = make_float2(i4.x, i4.y), bi1 = make_float2(i4.z, i4.w);
            re = __ffma2_rn(wai[p], bi0, __ffma2_rn(war[p], br0, re));
            ima = __ffma2_rn(wai[p], br0, ima);
            imb = __ffma2_rn(war[p], bi0, imb);
            re = __ffma2_rn(wai[p + 1], bi1, __ffma2_rn(war[p + 1], br1, re));
            ima = __ffma2_rn(wai[p + 1], br1, ima);
            imb = __ffma2_rn(war[p + 1], bi1, imb);
        }
        // both halves, in the same order for both threads of the pair
        float rs = hsum(re), is = hsum(ima) - hsum(imb);
        const float rs_o = __shfl_xor_sync(0xffffffffu, rs, 1), is_o = __shfl_xor_sync(0xffffffffu, is, 1);
        const float rv = (hh == 0 ? rs + rs_o : rs_o + rs) * inv_tr;
        const float iv = (hh == 0 ? is + is_o : is_o + is) * inv_tr;
        if (hh == 0) {
            const bool upper = arow < b;
            packed[arow * PK + b] = upper ? rv : iv;
            packed[b * PK + arow] = upper ? -iv : rv;
        }
    }
    if (t == 0) {   // the exact trace of the stored (normalised) diagonal, in row order
        float th = 0.0f, tl = 0.0f;
        for (int r = 0; r < D; ++r) {
            const float x = rowv[r] * inv_tr;
            const float sum = th + x, bp = sum - th;
            tl += (th - (sum - bp)) + (x - bp);
            th = sum;
        }
        a.trace_out[c] = (double)th + (double)tl;
    }
    __syncthreads();

    // ---- 5. store packed rho (FP32) -----------------------------------------------------------
    float *dst = a.rho_out + c * a.d_pad;
    for (int e = 4 * t; e < d; e += 4 * S::threads) {
        auto staged = [&](int ee) { return packed[(ee / D) * PK + (ee % D)]; };
        const float4 v = make_float4(staged(e), staged(e + 1), staged(e + 2), staged(e + 3));
        *reinterpret_cast<float4 *>(dst + e) = v;
        if (a.rho_norm_out) *reinterpret_cast<float4 *>(a.rho_norm_out + c * d + e) = v;
    }
}

template <int PASSES>
cudaError_t launch_propose_d64(const ProposeArgs &a, cudaStream_t s) {
    using S = Wide64;
    const size_t smem = sizeof(float) * S::smem_floats;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(propose_kernel_d64<PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(propose_kernel_d64<PASSES>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.rows <= 0) return cudaSuccess;
    propose_kernel_d64<PASSES><<<(unsigned)a.rows, S::threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int PASSES>
cudaError_t launch_propose_d32(const ProposeArgs &a, cudaStream_t s) {
    constexpr int THREADS = (PASSES == 3) ? 64 : kThreads;   // two chains per CTA with the refinement
    using S = WideShape<PASSES, THREADS>;
    const size_t smem = sizeof(float) * S::smem_floats * S::chains_per_block;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(propose_kernel_d32<PASSES, THREADS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(propose_kernel_d32<PASSES, THREADS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t blocks = (a.rows + S::chains_per_block - 1) / S::chains_per_block;
    if (blocks == 0) return cudaSuccess;
    propose_kernel_d32<PASSES, THREADS><<<(unsigned)blocks, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int D, int PASSES, int THREADS>
cudaError_t launch_propose_small(const ProposeArgs &a, int64_t rows, cudaStream_t s) {
    using S = Shape<D, PASSES, THREADS>;
    const size_t smem = sizeof(float) * S::smem_floats * S::chains_per_block;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(propose_kernel<D, PASSES, THREADS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(propose_kernel<D, PASSES, THREADS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t blocks = (rows + S::chains_per_block - 1) / S::chains_per_block;
    if (blocks == 0) return cudaSuccess;
    propose_kernel<D, PASSES, THREADS><<<(unsigned)blocks, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int D, int PASSES>
cudaError_t launch_propose_pd(const ProblemView &p, int mode, uint32_t step, const StepState *step_dev,
                              const float *x_eval, int64_t rows, bool want_split, float *rho_norm_out, cudaStream_t s) {
    ProposeArgs a;
    a.x_eval = x_eval;
    a.y = p.y;
    a.cur = p.cur;
    a.coef = p.coef;
    a.rho_out = p.rho_prop;
    a.split_out = (want_split && p.tc_kind == TC_BF16X3) ? static_cast<__nv_bfloat16 *>(p.rho_split) : nullptr;
    a.split_tf = (want_split && (p.tc_kind == TC_TF32 || p.tc_kind == TC_TF32X2)) ? static_cast<float *>(p.rho_split)
                                                                                   : nullptr;
    a.tf_splits = tc_splits(p.tc_kind);
    a.trace_out = p.trace_prop;
    a.rho_norm_out = (mode == MODE_EVAL) ? rho_norm_out : nullptr;
    a.rows = rows;
    a.R = p.R;
    a.chain_offset = p.chain_offset;
    a.seed = p.seed;
    a.rk = Philox::round_keys(p.seed);
    a.step = step;
    a.step_dev = step_dev;
    a.mode = mode;
    a.d_pad = p.d_pad;
    // the six-qubit kernel has no refinement: it takes the FP32 re-orthogonalisation
    constexpr int WIDE_PASSES = PASSES == 3 ? 2 : PASSES;
    if constexpr (D == 64) {
        if (a.split_out || a.split_tf) return cudaErrorNotSupported;   // no tensor-core form at D = 64
        return launch_propose_d64<WIDE_PASSES>(a, s);
    } else if constexpr (D == 32) {
        if (a.split_tf) return cudaErrorNotSupported;   // the TF32 forms stop at D = 16
        return launch_propose_d32<PASSES>(a, s);
    } else {
        // the CTA sizes the autotuner may pick are built for the default QR (3) and the
        // Hilbert-Schmidt prior (0); other settings run 128-thread CTAs
        if constexpr (PASSES == 0 || PASSES == 3) {
            if (p.propose_threads == 32) return launch_propose_small<D, PASSES, 32>(a, rows, s);
            if (p.propose_threads == 64) return launch_propose_small<D, PASSES, 64>(a, rows, s);
        }
        return launch_propose_small<D, PASSES, kThreads>(a, rows, s);
    }
}

template <int D>
cudaError_t launch_propose_d(const ProblemView &p, int mode, uint32_t step, const StepState *step_dev, const float *x_eval,
                             int64_t rows, bool want_split, float *rho_norm_out, cudaStream_t s) {
    if (p.qr_passes == 0) return launch_propose_pd<D, 0>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
    if (p.qr_passes == 1) return launch_propose_pd<D, 1>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
    if (p.qr_passes == 2) return launch_propose_pd<D, 2>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
    return launch_propose_pd<D, 3>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
}

}  // namespace

cudaError_t launch_propose(const ProblemView &p, int mode, uint32_t step, const StepState *step_dev, const float *x_eval,
                           int64_t n_eval, bool want_split, float *rho_norm_out, uint32_t *status, cudaStream_t s) {
    (void)status;
    const int64_t rows = (mode == MODE_EVAL) ? n_eval : p.R;
    switch (p.D) {
        case 2: return launch_propose_d<2>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
        case 4: return launch_propose_d<4>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
        case 8: return launch_propose_d<8>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
        case 16: return launch_propose_d<16>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
        case 32: return launch_propose_d<32>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
        case 64: return launch_propose_d<64>(p, mode, step, step_dev, x_eval, rows, want_split, rho_norm_out, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qst
