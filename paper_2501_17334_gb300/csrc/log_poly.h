/* Natural logarithm of a positive normal float, used by the likelihood epilogues.
 *
 * Method (the textbook reduction): x = 2^k m with m in [sqrt(1/2), sqrt(2)), so f = m - 1 is
 * exact and |f| <= 0.4143; log x = k ln2 + log1p(f) with log1p(f) = f + f^2 Q(f), Q a degree-8
 * polynomial fitted to (log1p(f) - f) / f^2 on that interval (log_poly_fit.py, beside this
 * file, reproduces the coefficients); ln2 is split so that k * LN2_HI is exact for |k| < 256.
 * Accuracy: at most 0.93 ulp on a sweep of 4e7 arguments from e^-20 to e^10 and around 1
 * (tests/test_log_poly.py), absolute error below 2.4e-8 for |x - 1| < 0.3.  Every operation is
 * an IEEE single-rounding one (fmaf), so host and device give identical bits.
 *
 * Callers pass x > 0 normal; x <= 0, denormals, inf and NaN are the caller's business (the
 * epilogues map p <= 0 to -inf themselves).  Valid as C99 and as CUDA host/device code.
 */
#ifndef QST_LOG_POLY_H
#define QST_LOG_POLY_H

#include <math.h>
#include <string.h>

#ifdef __CUDACC__
#define QST_LP_FN __host__ __device__ __forceinline__
#else
#define QST_LP_FN static inline
#endif

QST_LP_FN int qst_lp_bits(float x) {
    int i;
    memcpy(&i, &x, sizeof i);
    return i;
}
QST_LP_FN float qst_lp_float(int i) {
    float x;
    memcpy(&x, &i, sizeof x);
    return x;
}

QST_LP_FN float qst_log_poly(float x) {
    const int ix = qst_lp_bits(x);
    const int k = (ix - 0x3f3504f3) >> 23; /* 0x3f3504f3 = sqrt(1/2) */
    const float m = qst_lp_float(ix - (k << 23));
    const float f = m - 1.0f;
    const float kf = (float)k;
    float q = -0.08064694682313636f;
    q = fmaf(q, f, 0.1291790293475221f);
    q = fmaf(q, f, -0.13072555472249744f);
    q = fmaf(q, f, 0.14173450906326862f);
    q = fmaf(q, f, -0.16628919666247013f);
    q = fmaf(q, f, 0.20002695649848323f);
    q = fmaf(q, f, -0.25000751231191953f);
    q = fmaf(q, f, 0.33333312940994586f);
    q = fmaf(q, f, -0.49999997733204976f);
    const float f2 = f * f;
    const float r = fmaf(f2, q, fmaf(kf, 1.42860677e-06f, f)); /* LN2_LO = ln2 - LN2_HI */
    return fmaf(kf, 0.693145751953125f, r);                     /* LN2_HI = 0x1.62e4p-1 */
}

#endif
