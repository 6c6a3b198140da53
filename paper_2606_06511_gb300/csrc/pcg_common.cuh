// Shared device helpers of the PCG solvers: the dot-product accumulator (FP32 pairs for
// FP32 vectors) and the inverse of a regularised 3x3 block.
#pragma once
#include "common.cuh"

namespace ttie {

// Accumulator of dot products of T vectors and the arithmetic of the CG recurrence.  For FP32
// vectors it is an unevaluated sum of two floats (hi + lo, about 48 significant bits):
// products are split exactly with one fma and added with Knuth's two-sum, all at the FP32
// rate.  GB300 executes FP64 at a small fraction of the FP32 rate (a warp-wide FP64
// instruction occupies its pipe for tens of cycles), and a block-wide FP64 reduction per
// iteration costs microseconds.  For FP64 vectors it is a plain double.
template <typename T> struct Acc;
template <> struct Acc<double> {
    static constexpr int kTagShift = 0;   // a tag in bits() sits in the significand's lowest bits
    double v = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ void add(const Acc &o) { v += o.v; }
    __device__ __forceinline__ Acc shfl_xor(unsigned mask, int o, int width) const {
        Acc r;
        r.v = __shfl_xor_sync(mask, v, o, width);
        return r;
    }
    __device__ __forceinline__ unsigned long long bits() const { return (unsigned long long)__double_as_longlong(v); }
    __device__ __forceinline__ static Acc from_bits(unsigned long long b) {
        Acc r;
        r.v = __longlong_as_double((long long)b);
        return r;
    }
    __device__ __forceinline__ Acc times(double b) const { Acc r; r.v = v * b; return r; }
    __device__ __forceinline__ Acc over(double b) const { Acc r; r.v = v / b; return r; }
    __device__ __forceinline__ Acc minus(const Acc &o) const { Acc r; r.v = v - o.v; return r; }
    __device__ __forceinline__ double approx() const { return v; }
    __device__ __forceinline__ double value() const { return v; }
};
template <> struct Acc<float> {
    static constexpr int kTagShift = 32;  // a tag in bits() sits in the lowest bits of lo's significand
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_pair(float bh, float bl) {
        const float s = hi + bh, bb = s - hi;
        const float e = (hi - (s - bb)) + (bh - bb) + lo + bl;
        hi = s + e;
        lo = e - (hi - s);
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = a * b;
        add_pair(p, fmaf(a, b, -p));
    }
    __device__ __forceinline__ void add(const Acc &o) { add_pair(o.hi, o.lo); }
    __device__ __forceinline__ Acc shfl_xor(unsigned mask, int o, int width) const {
        Acc r;
        r.hi = __shfl_xor_sync(mask, hi, o, width);
        r.lo = __shfl_xor_sync(mask, lo, o, width);
        return r;
    }
    __device__ __forceinline__ unsigned long long bits() const {
        return (unsigned long long)__float_as_uint(hi) | ((unsigned long long)__float_as_uint(lo) << 32);
    }
    __device__ __forceinline__ static Acc from_bits(unsigned long long b) {
        Acc r;
        r.hi = __uint_as_float((unsigned)b);
        r.lo = __uint_as_float((unsigned)(b >> 32));
        return r;
    }
    __device__ __forceinline__ Acc times(float b) const {   // (hi + lo) b
        const float p = hi * b, e = fmaf(hi, b, -p) + lo * b;
        Acc r;
        r.hi = p + e;
        r.lo = e - (r.hi - p);
        return r;
    }
    __device__ __forceinline__ Acc over(float b) const {    // (hi + lo) / b, one correction step
        const float q1 = hi / b, p = q1 * b, pe = fmaf(q1, b, -p);
        const float q2 = (((hi - p) - pe) + lo) / b;
        Acc r;
        r.hi = q1 + q2;
        r.lo = q2 - (r.hi - q1);
        return r;
    }
    __device__ __forceinline__ Acc minus(const Acc &o) const {
        Acc r = *this;
        r.add_pair(-o.hi, -o.lo);
        return r;
    }
    __device__ __forceinline__ float approx() const { return hi + lo; }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Inverse of the 3x3 block m + mu I (row-major), by the adjugate.
template <typename T>
__device__ __forceinline__ void inv3(const T *m, T mu, T *o) {
    const double a = (double)m[0] + mu, b = m[1], c = m[2], d = m[3], e = (double)m[4] + mu, f = m[5], g = m[6], h = m[7],
                 i = (double)m[8] + mu;
    const double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
    const double det = a * A + b * B + c * C;
    const double id = det != 0.0 ? 1.0 / det : 0.0;
    o[0] = (T)(A * id); o[1] = (T)(-(b * i - c * h) * id); o[2] = (T)((b * f - c * e) * id);
    o[3] = (T)(B * id); o[4] = (T)((a * i - c * g) * id); o[5] = (T)(-(a * f - c * d) * id);
    o[6] = (T)(C * id); o[7] = (T)(-(a * h - b * g) * id); o[8] = (T)((a * e - b * d) * id);
}

// Chebyshev preconditioner (TTIE_PCG_CHEBYSHEV): block-Jacobi iterations before the estimate
// of lambda_max(D^-1 A), the margin on that estimate, lambda_max / lambda_min of the interval
// and the largest degree.
constexpr int kChebWarm = 6;
constexpr double kChebSafety = 1.1;
constexpr double kChebRatio = 10.0;
constexpr int kChebMaxDeg = 8;

// Eigenvalues below x of the symmetric tridiagonal (diagonal dg, squared off-diagonal e2):
// the number of negative pivots of its LDL^T factorisation shifted by x (Sturm sequence).
__device__ __forceinline__ int sturm_below(const double *dg, const double *e2, int m, double x) {
    int below = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
        q = dg[i] - x - (i ? e2[i - 1] / q : 0.0);
        if (q == 0.0) q = 1e-300;
        below += q < 0.0;
    }
    return below;
}

// From the first kChebWarm CG coefficients (al[j], be[j]: alpha and beta of iteration j; be[0]
// unused), the Lanczos tridiagonal of D^-1 A: diagonal 1/al[j] + be[j]/al[j-1], off-diagonal
// sqrt(be[j+1])/al[j].  Its largest eigenvalue (a lower bound of lambda_max, by bisection on
// the Sturm count from its Gershgorin bound) times kChebSafety is the interval's top; the
// Chebyshev iteration y = p_k(D^-1 A) D^-1 v on [top / kChebRatio, top] then runs
//   rr = D^-1 v,  d = rr / theta,  y = d;  for j < k: rr -= D^-1 A d,
//   d = c1[j] d + c2[j] rr,  y += d
// with theta, delta the interval's centre and half-width, sigma = theta / delta,
// rho_0 = 1 / sigma, rho_{j+1} = 1 / (2 sigma - rho_j), c1[j] = rho_{j+1} rho_j and
// c2[j] = 2 rho_{j+1} / delta.  Same inputs in every block, same coefficients.  False (keep
// block Jacobi) when a coefficient is not positive and finite.
template <typename T>
__device__ __noinline__ bool cheb_coefficients(const double *al, const double *be, int deg, T *c1, T *c2, T *theta_inv) {
    double dg[kChebWarm], e2[kChebWarm];
    for (int j = 0; j < kChebWarm; ++j) {
        if (!(al[j] > 0.0) || !isfinite(al[j]) || (j > 0 && (!(be[j] > 0.0) || !isfinite(be[j])))) return false;
        dg[j] = 1.0 / al[j] + (j ? be[j] / al[j - 1] : 0.0);
        if (j > 0) e2[j - 1] = be[j] / (al[j - 1] * al[j - 1]);
    }
    double hi = 0.0;
    for (int i = 0; i < kChebWarm; ++i)
        hi = fmax(hi, dg[i] + (i ? sqrt(e2[i - 1]) : 0.0) + (i + 1 < kChebWarm ? sqrt(e2[i]) : 0.0));
    if (!(hi > 0.0) || !isfinite(hi)) return false;
    double lo = 0.0;
    for (int s = 0; s < 60; ++s) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_below(dg, e2, kChebWarm, mid) < kChebWarm) lo = mid;
        else hi = mid;
    }
    const double top = hi * kChebSafety, bot = top / kChebRatio;
    const double th = 0.5 * (top + bot), de = 0.5 * (top - bot), sig = th / de;
    double rho = 1.0 / sig;
    for (int j = 0; j < deg; ++j) {
        const double rn = 1.0 / (2.0 * sig - rho);
        c1[j] = (T)(rn * rho);
        c2[j] = (T)(2.0 * rn / de);
        rho = rn;
    }
    *theta_inv = (T)(1.0 / th);
    return true;
}


}  // namespace ttie
