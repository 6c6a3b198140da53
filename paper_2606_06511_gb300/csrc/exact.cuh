// Exact sign of a 3x3 orientation determinant with floating-point expansions.
//
// Method: Shewchuk, "Adaptive Precision Floating-Point Arithmetic and Fast Robust
// Geometric Predicates" (1997): TWO-SUM, TWO-PRODUCT (here through fma),
// EXPANSION-SUM and SCALE-EXPANSION produce a non-overlapping expansion whose
// largest non-zero component has the sign of the exact value.  Written for this
// library; used only by the kernel that settles signs the floating-point
// filters could not certify.  Exact for inputs whose products neither
// overflow nor underflow (always the case for float32 inputs held in doubles).
#pragma once

namespace ttie {
namespace exact {

__device__ __forceinline__ void two_sum(double a, double b, double &x, double &y) {
    x = a + b;
    double bv = x - a;
    double av = x - bv;
    y = (a - av) + (b - bv);
}

// requires |a| >= |b| or a == 0
__device__ __forceinline__ void fast_two_sum(double a, double b, double &x, double &y) {
    x = a + b;
    y = b - (x - a);
}

__device__ __forceinline__ void two_prod(double a, double b, double &x, double &y) {
    x = a * b;
    y = fma(a, b, -x);
}

// h[0 .. m+n) = e[0 .. m) + f[0 .. n); every f component is grown into the running sum.
__device__ __forceinline__ int expansion_sum(int m, const double *e, int n, const double *f, double *h) {
    for (int i = 0; i < m; ++i) h[i] = e[i];
    for (int j = 0; j < n; ++j) {
        double q = f[j];
        for (int i = j; i < j + m; ++i) {
            double lo;
            two_sum(q, h[i], q, lo);
            h[i] = lo;
        }
        h[j + m] = q;
    }
    return m + n;
}

// h[0 .. 2m) = b * e[0 .. m)
__device__ __forceinline__ int scale_expansion(int m, const double *e, double b, double *h) {
    double q, t, tt;
    two_prod(e[0], b, q, h[0]);
    for (int i = 1; i < m; ++i) {
        two_prod(e[i], b, tt, t);
        two_sum(q, t, q, h[2 * i - 1]);
        fast_two_sum(tt, q, q, h[2 * i]);
    }
    h[2 * m - 1] = q;
    return 2 * m;
}

__device__ __forceinline__ int expansion_sign(int m, const double *e) {
    for (int i = m - 1; i >= 0; --i) {
        if (e[i] > 0.0) return 1;
        if (e[i] < 0.0) return -1;
    }
    return 0;
}

// px*qy - qx*py as a 4-component expansion
__device__ __forceinline__ void minor2(double px, double py, double qx, double qy, double *h) {
    double a[2], b[2];
    two_prod(px, qy, a[1], a[0]);
    two_prod(qx, py, b[1], b[0]);
    b[0] = -b[0];
    b[1] = -b[1];
    expansion_sum(2, a, 2, b, h);
}

// det [[px py 1] [qx qy 1] [rx ry 1]] = m(p,q) + m(q,r) + m(r,p): 12 components
__device__ __forceinline__ void det3xy1(const double *p, const double *q, const double *r, double *h) {
    double m1[4], m2[4], m3[4], s[8];
    minor2(p[0], p[1], q[0], q[1], m1);
    minor2(q[0], q[1], r[0], r[1], m2);
    minor2(r[0], r[1], p[0], p[1], m3);
    expansion_sum(4, m1, 4, m2, s);
    expansion_sum(8, s, 4, m3, h);
}

__device__ __forceinline__ void two_diff(double a, double b, double &x, double &y) {
    x = a - b;
    double bv = a - x;
    double av = x + bv;
    y = (a - av) + (bv - b);
}

// Sign of det[e1, e2, f] = e1 . (e2 x f) for exactly known entries: 24 components.
__device__ __noinline__ int det3_exact(const double *e1, const double *e2, const double *f) {
    double mx[4], my[4], mz[4], a[8], b[8], c[8], s16[16], s24[24];
    minor2(e2[1], e2[2], f[1], f[2], mx);   // e2y fz - fy e2z
    minor2(e2[2], e2[0], f[2], f[0], my);   // e2z fx - fz e2x
    minor2(e2[0], e2[1], f[0], f[1], mz);   // e2x fy - fx e2y
    scale_expansion(4, mx, e1[0], a);
    scale_expansion(4, my, e1[1], b);
    scale_expansion(4, mz, e1[2], c);
    expansion_sum(8, a, 8, b, s16);
    expansion_sum(16, s16, 8, c, s24);
    return expansion_sign(24, s24);
}

// Sign of det[e1, e2, f] for exactly known entries in integer arithmetic.  Scaled by 2^-lo,
// lo the exponent of the lowest set significand bit among the nine entries, every entry is
// an integer (exactly); when every scaled entry is below 2^40 in magnitude, the 2x2 minors
// (below 2^81) and the determinant (below 2^123) are exact in signed 128-bit integers.
// Entries of coordinate differences of float32 positions of similar magnitude have about 24
// to 30 significant bits and fit.  False (sign not set) for a subnormal, infinite or NaN
// entry, or entries whose bits span more than 40 places.
__device__ __forceinline__ bool det3_int_sign(const double *e1, const double *e2, const double *f, int &sign) {
    const double *rows[3] = {e1, e2, f};
    int lo = 1 << 20, hi = -(1 << 20);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double v = rows[r][k];
            if (v == 0.0) continue;
            const unsigned long long b = (unsigned long long)__double_as_longlong(v);
            const int E = (int)((b >> 52) & 0x7ff);
            if (E == 0 || E == 0x7ff) return false;
            const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
            lo = min(lo, E - 1075 + __ffsll((long long)m) - 1);   // lowest set bit: 2^lo
            hi = max(hi, E - 1023);                               // |v| < 2^(hi + 1)
        }
    if (hi < lo) { sign = 0; return true; }   // every entry zero
    if (hi - lo > 39) return false;
    long long I[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) I[r][k] = __double2ll_rn(ldexp(rows[r][k], -lo));
    const __int128 mx = (__int128)I[1][1] * I[2][2] - (__int128)I[1][2] * I[2][1];
    const __int128 my = (__int128)I[1][2] * I[2][0] - (__int128)I[1][0] * I[2][2];
    const __int128 mz = (__int128)I[1][0] * I[2][1] - (__int128)I[1][1] * I[2][0];
    const __int128 d = (__int128)I[0][0] * mx + (__int128)I[0][1] * my + (__int128)I[0][2] * mz;
    sign = (d > 0) - (d < 0);
    return true;
}

// ---- 256-bit two's-complement integers (arithmetic modulo 2^256; exact while the true
// values stay below 2^255 in magnitude)
struct I256 {
    unsigned long long w[4];
};
__device__ __forceinline__ I256 i256_from(__int128 v) {
    const unsigned long long ext = v < 0 ? ~0ull : 0ull;
    return {{(unsigned long long)v, (unsigned long long)(v >> 64), ext, ext}};
}
__device__ __forceinline__ I256 i256_add(const I256 &a, const I256 &b) {
    I256 r;
    unsigned long long c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned __int128 t = (unsigned __int128)a.w[k] + b.w[k] + c;
        r.w[k] = (unsigned long long)t;
        c = (unsigned long long)(t >> 64);
    }
    return r;
}
__device__ __forceinline__ I256 i256_neg(const I256 &a) {
    I256 r;
    unsigned long long c = 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned __int128 t = (unsigned __int128)(~a.w[k]) + c;
        r.w[k] = (unsigned long long)t;
        c = (unsigned long long)(t >> 64);
    }
    return r;
}
__device__ __forceinline__ I256 i256_mul(const I256 &a, const I256 &b) {
    I256 r = {{0ull, 0ull, 0ull, 0ull}};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long c = 0;
#pragma unroll
        for (int j = 0; i + j < 4; ++j) {
            const unsigned __int128 t = (unsigned __int128)a.w[i] * b.w[j] + r.w[i + j] + c;
            r.w[i + j] = (unsigned long long)t;
            c = (unsigned long long)(t >> 64);
        }
    }
    return r;
}
__device__ __forceinline__ int i256_sign(const I256 &a) {
    if ((long long)a.w[3] < 0) return -1;
    return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) ? 1 : 0;
}

// The 256-bit evaluation of orient3d_f32_int (coordinates spanning 40 to 79 bits), out of
// line so that the common 128-bit path stays small.
__device__ __noinline__ int orient3d_i256(const unsigned (&s)[4][3], const int (&ex)[4][3], const float *const (&P)[4],
                                          int lo) {
    __int128 X[4][3];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int sh = ex[p][k] - lo;
            __int128 v = sh >= 0 ? ((__int128)s[p][k] << sh) : (__int128)(s[p][k] >> (-sh));
            if (__float_as_uint(P[p][k]) >> 31) v = -v;
            X[p][k] = v;
        }
    I256 e1[3], e2[3], f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e1[k] = i256_from(X[1][k] - X[0][k]);
        e2[k] = i256_from(X[2][k] - X[0][k]);
        f[k] = i256_from(X[3][k] - X[0][k]);
    }
    // det = e1 . (e2 x f)
    const I256 mx = i256_add(i256_mul(e2[1], f[2]), i256_neg(i256_mul(e2[2], f[1])));
    const I256 my = i256_add(i256_mul(e2[2], f[0]), i256_neg(i256_mul(e2[0], f[2])));
    const I256 mz = i256_add(i256_mul(e2[0], f[1]), i256_neg(i256_mul(e2[1], f[0])));
    const I256 det = i256_add(i256_add(i256_mul(e1[0], mx), i256_mul(e1[1], my)), i256_mul(e1[2], mz));
    return i256_sign(det);
}

// Sign of det[b - a, c - a, d - a] for float32 points, in integer arithmetic.  Each coordinate
// is +-s 2^e with s < 2^24; scaled by 2^-lo (lo: the smallest exponent of a lowest set bit
// among the twelve) all are integers, below 2^(hi - lo + 1) with hi the largest exponent of a
// top bit.  When that bound is at most 2^39 the differences are below 2^40, the 2x2 minors
// below 2^81 and the determinant below 2^123: exact in 128-bit integers (coordinates of
// similar magnitude).  Up to 2^79: differences below 2^80, minors below 2^161, determinant
// below 2^243, exact in 256-bit integers (a mesh spanning 1e-17 to 10).  False (sign not set)
// for infinite or NaN coordinates or a wider span.
__device__ __noinline__ bool orient3d_f32_int(const float *a, const float *b, const float *c, const float *d,
                                              int &sign) {
    const float *P[4] = {a, b, c, d};
    unsigned s[4][3];
    int ex[4][3];
    int lo = 1 << 20, hi = -(1 << 20);
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const unsigned bits = __float_as_uint(P[p][k]);
            const int E = (int)((bits >> 23) & 0xffu);
            if (E == 255) return false;
            unsigned m = bits & 0x7fffffu;
            int e = -149;
            if (E != 0) {
                m |= 0x800000u;
                e = E - 150;
            }
            s[p][k] = m;
            ex[p][k] = e;
            if (m == 0) continue;
            lo = min(lo, e + __ffs((int)m) - 1);
            hi = max(hi, e + 31 - __clz((int)m));
        }
    if (hi < lo) { sign = 0; return true; }   // every coordinate zero
    if (hi - lo > 78) return false;
    // a right shift below drops only zero bits: lo is at most e + (trailing zeros of s)
    if (hi - lo <= 38) {
        long long X[4][3];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int sh = ex[p][k] - lo;
                long long v = sh >= 0 ? ((long long)s[p][k] << sh) : (long long)(s[p][k] >> (-sh));
                X[p][k] = (__float_as_uint(P[p][k]) >> 31) ? -v : v;
            }
        long long e1[3], e2[3], f[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            e1[k] = X[1][k] - X[0][k];
            e2[k] = X[2][k] - X[0][k];
            f[k] = X[3][k] - X[0][k];
        }
        const __int128 mx = (__int128)e2[1] * f[2] - (__int128)e2[2] * f[1];
        const __int128 my = (__int128)e2[2] * f[0] - (__int128)e2[0] * f[2];
        const __int128 mz = (__int128)e2[0] * f[1] - (__int128)e2[1] * f[0];
        const __int128 det = (__int128)e1[0] * mx + (__int128)e1[1] * my + (__int128)e1[2] * mz;
        sign = (det > 0) - (det < 0);
        return true;
    }
    sign = orient3d_i256(s, ex, P, lo);
    return true;
}

// Sign of det[b - a, c - a, d - a] (positive when d lies on the side of the plane
// (a, b, c) that the normal (b - a) x (c - a) points to).  When the nine coordinate
// differences are exact doubles (always the case for float32 inputs of similar
// magnitude) the 3x3 determinant of the differences is expanded directly; otherwise
// the 4x4 determinant with rows (x, y, z, 1) of a, b, c, d, which expanded along z
// equals -det[b - a, c - a, d - a].
__device__ __noinline__ int orient3d_exact(const double *a, const double *b, const double *c, const double *d) {
    double e1[3], e2[3], f[3], r1, r2, r3;
    bool exact_diff = true;
    for (int k = 0; k < 3; ++k) {
        two_diff(b[k], a[k], e1[k], r1);
        two_diff(c[k], a[k], e2[k], r2);
        two_diff(d[k], a[k], f[k], r3);
        exact_diff &= (r1 == 0.0) && (r2 == 0.0) && (r3 == 0.0);
    }
    if (exact_diff) return det3_exact(e1, e2, f);
    double t12[12], s24a[24], s24b[24], s48a[48], s48b[48], s96[96];
    det3xy1(b, c, d, t12);
    scale_expansion(12, t12, a[2], s24a);
    det3xy1(a, c, d, t12);
    scale_expansion(12, t12, -b[2], s24b);
    expansion_sum(24, s24a, 24, s24b, s48a);
    det3xy1(a, b, d, t12);
    scale_expansion(12, t12, c[2], s24a);
    det3xy1(a, b, c, t12);
    scale_expansion(12, t12, -d[2], s24b);
    expansion_sum(24, s24a, 24, s24b, s48b);
    expansion_sum(48, s48a, 48, s48b, s96);
    return -expansion_sign(96, s96);
}

}  // namespace exact
}  // namespace ttie
