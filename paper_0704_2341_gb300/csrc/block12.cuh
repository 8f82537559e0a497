// Inverse of one 12 x 12 complex block (spin x colour) in FP64, by
// Gauss-Jordan elimination with partial pivoting, in one thread: the
// site-block inverses of the Section 3 approximation (the diagonal d and the
// block row sums d~ of a rest-set operator).
#pragma once

#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ double2 b12_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// A is destroyed; B receives A^-1.  Returns false if a pivot is zero or not
// finite (B is then undefined).
__device__ inline bool invert12(double2 (&A)[12][12], double2 (&B)[12][12]) {
    for (int r = 0; r < 12; ++r)
        for (int q = 0; q < 12; ++q) B[r][q] = make_double2(r == q ? 1.0 : 0.0, 0.0);
    for (int c = 0; c < 12; ++c) {
        int piv = c;
        double best = A[c][c].x * A[c][c].x + A[c][c].y * A[c][c].y;
        for (int r = c + 1; r < 12; ++r) {
            const double m = A[r][c].x * A[r][c].x + A[r][c].y * A[r][c].y;
            if (m > best) {
                best = m;
                piv = r;
            }
        }
        if (!(best > 0.0) || !isfinite(best)) return false;
        if (piv != c)
            for (int q = 0; q < 12; ++q) {
                const double2 ta = A[c][q], tb = B[c][q];
                A[c][q] = A[piv][q];
                B[c][q] = B[piv][q];
                A[piv][q] = ta;
                B[piv][q] = tb;
            }
        const double2 pv = A[c][c];
        const double inv = 1.0 / best;
        const double2 rp = make_double2(pv.x * inv, -pv.y * inv);   // 1 / pivot
        for (int q = 0; q < 12; ++q) {
            A[c][q] = b12_mul(A[c][q], rp);
            B[c][q] = b12_mul(B[c][q], rp);
        }
        for (int r = 0; r < 12; ++r) {
            if (r == c) continue;
            const double2 f = A[r][c];
            if (f.x == 0.0 && f.y == 0.0) continue;
            for (int q = 0; q < 12; ++q) {
                const double2 ua = b12_mul(f, A[c][q]), ub = b12_mul(f, B[c][q]);
                A[r][q].x -= ua.x;
                A[r][q].y -= ua.y;
                B[r][q].x -= ub.x;
                B[r][q].y -= ub.y;
            }
        }
    }
    return true;
}

}  // namespace gs
