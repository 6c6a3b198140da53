/*
 * TTIE oracle, per-pair core.  TEST INFRASTRUCTURE ONLY: this file is part of the
 * CPU oracle that checks the CUDA path.  The product never links or calls it.
 *
 * Plain FP64.  Forward-mode dual numbers carry d/dx of every intermediate with
 * respect to the 18 coordinates of the pair, the way the paper obtains its
 * derivatives for clarity (Appendix A, "C++ Code for our 3DTTI energy"; §1.2
 * says the autodiff form is the reference for the hand-built GPU graph).
 *
 * Pair layout: loc = [A0 A1 A2 B0 B1 B2] (xyz each), A = first triangle of the
 * pair (u_0..2 in §1), B = second (v_0..2).  The appendix stores the same
 * 18-vector with the first triangle first.
 *
 * Steps (§1, Eq. 1 and Appendix A):
 *   1. plane_cut(P, Q): n = normalize((P1-P0) x (P2-P0)); d_k = n.(Q_k - P_k).
 *      Q straddles the plane of P iff some d_k > 0 and some d_k < 0.  The cut
 *      segment runs between the crossings of the two edges that leave the vertex
 *      whose sign is unique; when one d_k is exactly 0 (signs +,-,0) it runs from
 *      that vertex to the crossing of the opposite edge.
 *   2. segment on B from the plane of A, segment on A from the plane of B.
 *   3. D = normalize(n_B x n_A) with unnormalised normals (the appendix's
 *      uNormal x vNormal with U the second triangle).
 *   4. origin O = mean of the four segment endpoints; t = D.(S - O).
 *   5. I_A = [min, max] of A's two t, I_B likewise;
 *      t_c^0 = s (t_A^0 - t_B^1),  t_c^1 = s (t_A^1 - t_B^0)   (Eq. 1, s = 1;
 *      the appendix's listing multiplies by s = 1/2).
 *   6. FP64 overlap flag: t_A^1 > t_B^0 and t_A^0 < t_B^1 (the open criterion
 *      0 in (t_c^0, t_c^1) of §1).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NX 18

typedef struct { double v; double g[NX]; } dual;
typedef struct { dual c[3]; } dvec;

static dual d_const(double v) { dual r; r.v = v; memset(r.g, 0, sizeof r.g); return r; }
static dual d_add(dual a, dual b) { dual r; r.v = a.v + b.v; for (int i = 0; i < NX; ++i) r.g[i] = a.g[i] + b.g[i]; return r; }
static dual d_sub(dual a, dual b) { dual r; r.v = a.v - b.v; for (int i = 0; i < NX; ++i) r.g[i] = a.g[i] - b.g[i]; return r; }
static dual d_mul(dual a, dual b) {
    dual r; r.v = a.v * b.v;
    for (int i = 0; i < NX; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
    return r;
}
static dual d_div(dual a, dual b) {
    dual r; r.v = a.v / b.v;
    for (int i = 0; i < NX; ++i) r.g[i] = (a.g[i] * b.v - a.v * b.g[i]) / (b.v * b.v);
    return r;
}
static dual d_scale(dual a, double s) { dual r; r.v = a.v * s; for (int i = 0; i < NX; ++i) r.g[i] = a.g[i] * s; return r; }
static dual d_sqrt(dual a) {
    dual r; r.v = sqrt(a.v);
    for (int i = 0; i < NX; ++i) r.g[i] = a.g[i] / (2.0 * r.v);
    return r;
}

static dvec v_sub(dvec a, dvec b) { dvec r; for (int k = 0; k < 3; ++k) r.c[k] = d_sub(a.c[k], b.c[k]); return r; }
static dvec v_add(dvec a, dvec b) { dvec r; for (int k = 0; k < 3; ++k) r.c[k] = d_add(a.c[k], b.c[k]); return r; }
static dvec v_mul(dvec a, dual s) { dvec r; for (int k = 0; k < 3; ++k) r.c[k] = d_mul(a.c[k], s); return r; }
static dvec v_div(dvec a, dual s) { dvec r; for (int k = 0; k < 3; ++k) r.c[k] = d_div(a.c[k], s); return r; }
static dvec v_scale(dvec a, double s) { dvec r; for (int k = 0; k < 3; ++k) r.c[k] = d_scale(a.c[k], s); return r; }
static dual v_dot(dvec a, dvec b) {
    return d_add(d_add(d_mul(a.c[0], b.c[0]), d_mul(a.c[1], b.c[1])), d_mul(a.c[2], b.c[2]));
}
static dvec v_cross(dvec a, dvec b) {
    dvec r;
    r.c[0] = d_sub(d_mul(a.c[1], b.c[2]), d_mul(a.c[2], b.c[1]));
    r.c[1] = d_sub(d_mul(a.c[2], b.c[0]), d_mul(a.c[0], b.c[2]));
    r.c[2] = d_sub(d_mul(a.c[0], b.c[1]), d_mul(a.c[1], b.c[0]));
    return r;
}
static dvec v_normalize(dvec a) { return v_div(a, d_sqrt(v_dot(a, a))); }

/* Point where the edge (Qm, Qp) meets the plane, from the signed distances dm, dp
 * of its ends: (dp Qm - dm Qp) / (dp - dm). */
static dvec crossing(dvec Qm, dual dm, dvec Qp, dual dp) {
    return v_div(v_sub(v_mul(Qm, dp), v_mul(Qp, dm)), d_sub(dp, dm));
}

/* Cut triangle Q by the plane of triangle P.  Returns 1 and the segment (s0, s1)
 * when Q straddles the plane; sgn[k] receives the FP64 side of Q_k. */
static int plane_cut(const dvec P[3], const dvec Q[3], dvec *s0, dvec *s1, int sgn[3]) {
    dvec n = v_normalize(v_cross(v_sub(P[1], P[0]), v_sub(P[2], P[0])));
    dual d[3];
    int pos = 0, neg = 0;
    for (int k = 0; k < 3; ++k) {
        d[k] = v_dot(n, v_sub(Q[k], P[k]));
        sgn[k] = d[k].v > 0.0 ? 1 : (d[k].v < 0.0 ? -1 : 0);
        pos += sgn[k] > 0;
        neg += sgn[k] < 0;
    }
    if (!(pos > 0 && neg > 0)) return 0;
    if (pos + neg == 2) {
        /* signs {+,-,0}: segment from the on-plane vertex to the crossing of the opposite edge */
        int z = sgn[0] == 0 ? 0 : (sgn[1] == 0 ? 1 : 2);
        int p = (z + 1) % 3, q = (z + 2) % 3;
        if (p > q) { int t = p; p = q; q = t; }
        *s0 = Q[z];
        *s1 = crossing(Q[p], d[p], Q[q], d[q]);
    } else {
        /* signs 2:1: the edges leaving the vertex with the unique sign */
        int lone_sign = (pos == 1) ? 1 : -1;
        int m = sgn[0] == lone_sign ? 0 : (sgn[1] == lone_sign ? 1 : 2);
        int p = (m + 1) % 3, q = (m + 2) % 3;
        if (p > q) { int t = p; p = q; q = t; }
        *s0 = crossing(Q[m], d[m], Q[p], d[p]);
        *s1 = crossing(Q[m], d[m], Q[q], d[q]);
    }
    return 1;
}

static dual d_min(dual a, dual b) { return (b.v < a.v) ? b : a; }
static dual d_max(dual a, dual b) { return (b.v > a.v) ? b : a; }

/* One pair.  loc[18] = [A0 A1 A2 B0 B1 B2].  Outputs:
 *   tc[2]      t_c^0, t_c^1 (zero when a triangle does not straddle)
 *   grad[36]   d t_c^0 / d loc (18), then d t_c^1 / d loc (18)
 *   sgn[6]     FP64 sides of B's vertices w.r.t. plane A, then A's w.r.t. plane B
 * Returns flags: bit0 B straddles plane A, bit1 A straddles plane B,
 *                bit2 FP64 open-interval overlap (both straddle and 0 in (t_c^0, t_c^1)). */
static int oracle_pair(const double loc[NX], double tc_scale, double tc[2], double grad[36], int sgn[6]) {
    dvec A[3], B[3];
    for (int v = 0; v < 3; ++v)
        for (int k = 0; k < 3; ++k) {
            A[v].c[k] = d_const(loc[3 * v + k]);
            A[v].c[k].g[3 * v + k] = 1.0;
            B[v].c[k] = d_const(loc[9 + 3 * v + k]);
            B[v].c[k].g[9 + 3 * v + k] = 1.0;
        }
    dvec sB0, sB1, sA0, sA1;
    int flags = 0;
    if (plane_cut(A, B, &sB0, &sB1, sgn)) flags |= 1;
    if (plane_cut(B, A, &sA0, &sA1, sgn + 3)) flags |= 2;
    tc[0] = tc[1] = 0.0;
    memset(grad, 0, 36 * sizeof(double));
    if (flags != 3) return flags;

    dvec nA = v_cross(v_sub(A[1], A[0]), v_sub(A[2], A[0]));
    dvec nB = v_cross(v_sub(B[1], B[0]), v_sub(B[2], B[0]));
    dvec D = v_normalize(v_cross(nB, nA));
    dvec O = v_scale(v_add(v_add(sA0, sA1), v_add(sB0, sB1)), 0.25);
    dual tA0 = v_dot(D, v_sub(sA0, O)), tA1 = v_dot(D, v_sub(sA1, O));
    dual tB0 = v_dot(D, v_sub(sB0, O)), tB1 = v_dot(D, v_sub(sB1, O));
    dual a_lo = d_min(tA0, tA1), a_hi = d_max(tA0, tA1);
    dual b_lo = d_min(tB0, tB1), b_hi = d_max(tB0, tB1);
    dual c0 = d_scale(d_sub(a_lo, b_hi), tc_scale);
    dual c1 = d_scale(d_sub(a_hi, b_lo), tc_scale);
    if (a_hi.v > b_lo.v && a_lo.v < b_hi.v) flags |= 4;
    tc[0] = c0.v;
    tc[1] = c1.v;
    for (int i = 0; i < NX; ++i) { grad[i] = c0.g[i]; grad[NX + i] = c1.g[i]; }
    return flags;
}

/* Batched entry: pairs[2p], pairs[2p+1] index triangles of tri (F x 3), x is V x 3. */
int ttie_oracle_eval(const double *x, const int32_t *tri, const int64_t *pairs, int64_t n_pairs,
                     double tc_scale, double *tc, double *grad, int8_t *sgn, uint8_t *flags) {
    for (int64_t p = 0; p < n_pairs; ++p) {
        double loc[NX];
        const int32_t *ta = tri + 3 * pairs[2 * p], *tb = tri + 3 * pairs[2 * p + 1];
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) {
                loc[3 * v + k] = x[3 * (int64_t)ta[v] + k];
                loc[9 + 3 * v + k] = x[3 * (int64_t)tb[v] + k];
            }
        int s[6];
        flags[p] = (uint8_t)oracle_pair(loc, tc_scale, tc + 2 * p, grad + 36 * p, s);
        for (int k = 0; k < 6; ++k) sgn[6 * p + k] = (int8_t)s[k];
    }
    return 0;
}

/*
 * Certified FP64 plane-side filter (not part of the paper's method: it only lets
 * the exact evaluation skip pairs whose census is certain).
 *
 * side(P, q) = det[P1-P0, P2-P0, q-P0], whose sign is the side of q w.r.t. the
 * plane of P (the normalised d_k above differs by a positive factor).  With
 * rounding unit u = 2^-53 the computed value differs from the exact one by at
 * most about 8u times the permanent (the same sum with every product taken in
 * absolute value); the filter trusts a sign only when |det| > 2e-15 * permanent
 * (about 18u).  Result per vertex: +1 / -1 certain, 2 uncertain.
 */
static int filtered_side(const double *P0, const double *P1, const double *P2, const double *q) {
    double e1[3], e2[3], f[3];
    for (int k = 0; k < 3; ++k) { e1[k] = P1[k] - P0[k]; e2[k] = P2[k] - P0[k]; f[k] = q[k] - P0[k]; }
    double m0 = e1[1] * e2[2] - e1[2] * e2[1];
    double m1 = e1[2] * e2[0] - e1[0] * e2[2];
    double m2 = e1[0] * e2[1] - e1[1] * e2[0];
    double det = m0 * f[0] + m1 * f[1] + m2 * f[2];
    double perm = (fabs(e1[1] * e2[2]) + fabs(e1[2] * e2[1])) * fabs(f[0])
                + (fabs(e1[2] * e2[0]) + fabs(e1[0] * e2[2])) * fabs(f[1])
                + (fabs(e1[0] * e2[1]) + fabs(e1[1] * e2[0])) * fabs(f[2]);
    double bound = 2e-15 * perm;
    if (!(perm > 1e-280)) return 2;
    if (det > bound) return 1;
    if (det < -bound) return -1;
    return 2;
}

/* For each pair: out[6p+k] = filtered side of B_k w.r.t. plane A (k<3), of A_{k-3}
 * w.r.t. plane B (k>=3). */
int ttie_oracle_sides(const double *x, const int32_t *tri, const int64_t *pairs, int64_t n_pairs, int8_t *out) {
    for (int64_t p = 0; p < n_pairs; ++p) {
        const int32_t *ta = tri + 3 * pairs[2 * p], *tb = tri + 3 * pairs[2 * p + 1];
        const double *A0 = x + 3 * (int64_t)ta[0], *A1 = x + 3 * (int64_t)ta[1], *A2 = x + 3 * (int64_t)ta[2];
        const double *B0 = x + 3 * (int64_t)tb[0], *B1 = x + 3 * (int64_t)tb[1], *B2 = x + 3 * (int64_t)tb[2];
        out[6 * p + 0] = (int8_t)filtered_side(A0, A1, A2, B0);
        out[6 * p + 1] = (int8_t)filtered_side(A0, A1, A2, B1);
        out[6 * p + 2] = (int8_t)filtered_side(A0, A1, A2, B2);
        out[6 * p + 3] = (int8_t)filtered_side(B0, B1, B2, A0);
        out[6 * p + 4] = (int8_t)filtered_side(B0, B1, B2, A1);
        out[6 * p + 5] = (int8_t)filtered_side(B0, B1, B2, A2);
    }
    return 0;
}
