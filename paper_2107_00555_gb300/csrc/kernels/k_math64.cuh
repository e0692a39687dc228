// k_math64.cuh -- binary64 exp, sin and cos for the fused kernels.
//
// A GB300 SM issues binary64 arithmetic at 1/64 of its binary32 rate, so a
// fused map over doubles that calls exp or sin is bound by its count of
// binary64 instructions, not by HBM.  These routines take the arguments of
// their fast paths with few binary64 operations (exp 10, sin / cos 15; the
// table index, the quadrant, the exponent scaling and the range tests are
// integer work) and hand every other argument -- large, non-finite, or with
// a result near overflow or underflow -- to CUDA's exp / sin / cos.
//
//   exp (Tang's table-driven method, ACM TOMS 15(2), 1989): x = k ln2/64 + r
//     with k = rint(64 x / ln2), |r| <= ln2/128 + rounding, ln2/64 in two
//     parts (Cody and Waite).  With k = 64 m + j, e^x = 2^m 2^(j/64) e^r;
//     e^r - 1 is its Taylor series to r^5, 2^(j/64) comes from a 64-entry
//     table, and 2^m is added to the exponent field.  The first dropped
//     term, r^6/6!, is at most (ln2/128)^6/720 = 2^-54.7 relative to e^r:
//     0.16 to 0.32 ulp of the result, the largest term of the error budget
//     after the final rounding.  Fast path |x| < 704, where 2^m 2^(j/64) e^r
//     is a normal double and the exponent addition cannot overflow.
//   sin, cos: x = k pi/2 + r with k = rint(2x/pi) and pi/2 in three parts
//     (Cody and Waite), |r| <= pi/4 + rounding; sin(x + q pi/2) is
//     +-sin r or +-cos r by (k + q) mod 4, with the Taylor series of sin r
//     to r^17 and of cos r to r^16.  The first dropped terms are at most
//     (pi/4)^19/19! = 2^-62.9 relative to sin r and (pi/4)^18/18! =
//     2^-58.3 relative to cos r (0.03 ulp), both at |r| = pi/4.  For
//     |x| < 2^17 the first part's product is cancelled exactly and the
//     three parts leave an error far below the rounding of r.  Fast path
//     |x| < 2^17.
//
// Error budget of the fast paths: the final rounding (0.5 ulp), the table
// entry and the rounding of r (each below 0.5 ulp of their own, scaled by
// the derivative), and the truncations above.  Measured: at most 1.2 ulp
// (exp) and 1.4 ulp (sin, cos) against 120-bit values; tests compare with
// the host's libm over the fast ranges, across the range limits and at the
// special values.
//
// Rounding is explicit (__fma_rn, __dmul_rn, __dsub_rn), so the results do
// not depend on the compiler's contraction choices.

// BEGIN generated by gen_math64_constants.py
#define DCP_M64_EXP_TAB 0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0, 0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0, 0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0, 0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0, 0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0, 0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0, 0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0, 0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0, 0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0, 0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0, 0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0, 0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0, 0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0, 0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0, 0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0, 0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0
#define DCP_M64_INV_L 0x1.71547652b82fep+6
#define DCP_M64_L 0x1.62e42fefa39efp-7, 0x1.abc9e3b39803fp-62
#define DCP_M64_TWO_OVER_PI 0x1.45f306dc9c883p-1
#define DCP_M64_PIO2 0x1.921fb54442d18p+0, 0x1.1a62633145c07p-54, -0x1.f1976b7ed8fbcp-110
#define DCP_M64_EXPM1_TAYLOR 0x1.0000000000000p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5, 0x1.1111111111111p-7
#define DCP_M64_SIN_TAYLOR -0x1.5555555555555p-3, 0x1.1111111111111p-7, -0x1.a01a01a01a01ap-13, 0x1.71de3a556c734p-19, -0x1.ae64567f544e4p-26, 0x1.6124613a86d09p-33, -0x1.ae7f3e733b81fp-41, 0x1.952c77030ad4ap-49
#define DCP_M64_COS_TAYLOR -0x1.0000000000000p-1, 0x1.5555555555555p-5, -0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-16, -0x1.27e4fb7789f5cp-22, 0x1.1eed8eff8d898p-29, -0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-45
// END generated by gen_math64_constants.py

// 2^(j/64) for j = 0..63 in device memory (read through the read-only path;
// 512 bytes, resident in L1 after the first touches).
__device__ double dcp_m64_exp_tab[64] = {DCP_M64_EXP_TAB};

// High word of |x|, for the range tests.
__device__ __forceinline__ unsigned dcp_m64_ahi(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
}

__device__ __forceinline__ double dcp_exp64(double x) {
  if (dcp_m64_ahi(x) < 0x40860000u) {  // |x| < 704
    // rint(64 x / ln2) by the 1.5 * 2^52 shifter: the sum's low word is k
    const double shifter = 0x1.8p52;
    const double t = __fma_rn(x, DCP_M64_INV_L, shifter);
    const int k = __double2loint(t);
    const double kf = __dsub_rn(t, shifter);
    const double l[2] = {DCP_M64_L};
    double r = __fma_rn(-kf, l[0], x);  // exact: x and k l[0] cancel
    r = __fma_rn(-kf, l[1], r);
    // e^r - 1 = r + r^2 (1/2! + r (1/3! + r (1/4! + r / 5!)))
    const double c[4] = {DCP_M64_EXPM1_TAYLOR};
    double p = __fma_rn(r, c[3], c[2]);
    p = __fma_rn(r, p, c[1]);
    p = __fma_rn(r, p, c[0]);
    const double em1 = __fma_rn(__dmul_rn(r, r), p, r);
    const double tj = __ldg(dcp_m64_exp_tab + (k & 63));
    const double y = __fma_rn(tj, em1, tj);
    // times 2^m, m = floor(k / 64): y stays normal on the fast path
    const unsigned long long m = (unsigned long long)(long long)(k >> 6);
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(y) + (m << 52)));
  }
  return exp(x);
}

// sin(x + q pi/2) for |x| < 2^17 (q = 0: sin, q = 1: cos).
__device__ __forceinline__ double dcp_sin_q64(double x, int q) {
  const double shifter = 0x1.8p52;
  const double t = __fma_rn(x, DCP_M64_TWO_OVER_PI, shifter);
  const int k = __double2loint(t) + q;
  const double kf = __dsub_rn(t, shifter);
  const double pio2[3] = {DCP_M64_PIO2};
  double r = __fma_rn(-kf, pio2[0], x);  // exact for |x| < 2^17
  r = __fma_rn(-kf, pio2[1], r);
  r = __fma_rn(-kf, pio2[2], r);
  // odd k: cos r = 1 + z P_c(z); even k: sin r = r + r z P_s(z); z = r^2
  const double cs[8] = {DCP_M64_SIN_TAYLOR};
  const double cc[8] = {DCP_M64_COS_TAYLOR};
  const bool odd = (k & 1) != 0;
  const double z = __dmul_rn(r, r);
  double p = odd ? cc[7] : cs[7];
#pragma unroll
  for (int i = 6; i >= 0; --i) p = __fma_rn(z, p, odd ? cc[i] : cs[i]);
  const double y = __fma_rn(odd ? z : __dmul_rn(r, z), p, odd ? 1.0 : r);
  // (k mod 4) in {2, 3}: negate
  return __longlong_as_double(__double_as_longlong(y) ^ ((long long)(k & 2) << 62));
}

__device__ __forceinline__ double dcp_sin64(double x) {
  const unsigned h = dcp_m64_ahi(x);
  if (h < 0x41000000u)  // |x| < 2^17; sin(+-0) keeps the sign of zero
    return (__double_as_longlong(x) << 1) == 0 ? x : dcp_sin_q64(x, 0);
  return sin(x);
}

__device__ __forceinline__ double dcp_cos64(double x) {
  if (dcp_m64_ahi(x) < 0x41000000u) return dcp_sin_q64(x, 1);  // |x| < 2^17
  return cos(x);
}
