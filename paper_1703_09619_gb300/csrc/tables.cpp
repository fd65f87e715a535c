// Host tables of libp2s: Gauss-Legendre rules and Legendre linearisation coefficients.
//
// Linearisation (Eq. (3) of arXiv:1703.09619 for the Legendre basis):
//   P_m P_n = sum_{r=0}^{min(m,n)} A_{m-r} A_r A_{n-r} / A_{m+n-r}
//             * (2m+2n-4r+1) / (2m+2n-2r+1) * P_{m+n-2r},   A_r = (2r-1)!! / r!
// (Adams' product formula), and for the derivative types the expansion
//   P'_m = sum_{j = m-1, m-3, ... >= 0} (2j+1) P_j,
// so dv, vd and dd coefficients are sums of Adams products.  Every nonzero
// coefficient of P^{(d1)}_{m1} P^{(d2)}_{m2} sits at k = m1+m2-d1-d2-2r, so each
// (type, m1, m2) is stored as a contiguous run k = kmin, kmin+2, ..., kmax.
//
// Gauss-Legendre rules: Newton's method on P_G in long double, started from the
// Tricomi asymptotic node estimate; weights 2 / ((1 - x^2) P'_G(x)^2).  The rule is
// symmetric (P_G has parity G): the non-negative roots are computed and mirrored, the
// middle node of an odd rule is exactly 0, so x[G-1-a] = -x[a] and w[G-1-a] = w[a] hold
// bit for bit (the double-word moment kernel folds its sums on that symmetry).
#include <cmath>
#include <cstring>
#include <mutex>

#include "p2s_internal.h"

namespace p2s {
namespace {

long double adams_A(int r) {
    long double a = 1.0L;
    for (int i = 1; i <= r; ++i) a *= (long double)(2 * i - 1) / (long double)i;
    return a;
}

// dense[k] += scale * coefficients of P_m P_n
void add_adams(int m, int n, long double scale, long double* dense) {
    int mn = m < n ? m : n;
    for (int r = 0; r <= mn; ++r) {
        long double c = adams_A(m - r) * adams_A(r) * adams_A(n - r) / adams_A(m + n - r) *
                        (long double)(2 * m + 2 * n - 4 * r + 1) / (long double)(2 * m + 2 * n - 2 * r + 1);
        dense[m + n - 2 * r] += scale * c;
    }
}

void product_dense(int d1, int d2, int m1, int m2, long double* dense /* [2*kMaxOrder] */) {
    for (int k = 0; k < 2 * kMaxOrder; ++k) dense[k] = 0.0L;
    // left factor: P_m1 or sum_j (2j+1) P_j ; right factor likewise
    int jl0 = d1 ? m1 - 1 : m1, jr0 = d2 ? m2 - 1 : m2;
    for (int jl = jl0; jl >= 0; jl -= 2) {
        long double cl = d1 ? (long double)(2 * jl + 1) : 1.0L;
        for (int jr = jr0; jr >= 0; jr -= 2) {
            long double cr = d2 ? (long double)(2 * jr + 1) : 1.0L;
            add_adams(jl, jr, cl * cr, dense);
            if (!d2) break;
        }
        if (!d1) break;
    }
}

void legendre_ld(int n, long double x, long double* p_n, long double* p_nm1) {
    long double p0 = 1.0L, p1 = x;
    if (n == 0) { *p_n = 1.0L; *p_nm1 = 0.0L; return; }
    for (int j = 1; j < n; ++j) {
        long double p2 = ((2 * j + 1) * x * p1 - j * p0) / (long double)(j + 1);
        p0 = p1;
        p1 = p2;
    }
    *p_n = p1;
    *p_nm1 = p0;
}

void gauss_legendre_ld(int G, double* x, double* w) {
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 1; i <= (G + 1) / 2; ++i) {
        // Tricomi estimate of the i-th largest root
        long double th = pi * (4.0L * i - 1.0L) / (4.0L * G + 2.0L);
        long double z = (1.0L - (G - 1.0L) / (8.0L * G * G * G)) * cosl(th);
        long double dp = 1.0L;
        for (int it = 0; it < 60; ++it) {
            long double pn, pm;
            legendre_ld(G, z, &pn, &pm);
            dp = G * (z * pn - pm) / (z * z - 1.0L);
            long double dz = pn / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        if (2 * i - 1 == G) z = 0.0L;  // the middle node of an odd rule
        long double pn, pm;
        legendre_ld(G, z, &pn, &pm);
        dp = G * (z * pn - pm) / (z * z - 1.0L);
        const double xd = (double)z, wd = (double)(2.0L / ((1.0L - z * z) * dp * dp));
        x[G - i] = xd;
        w[G - i] = wd;
        x[i - 1] = -xd;
        w[i - 1] = wd;
    }
}

HostTables* build() {
    static HostTables T;
    std::memset(&T, 0, sizeof(T));
    for (int G = 1; G <= kMaxG; ++G) gauss_legendre_ld(G, T.gl_x[G], T.gl_w[G]);
    int off = 0;
    long double dense[2 * kMaxOrder];
    for (int t = 0; t < kNumTypes; ++t) {
        int d1 = t & 1, d2 = (t >> 1) & 1;
        for (int m1 = 0; m1 < kMaxOrder; ++m1)
            for (int m2 = 0; m2 < kMaxOrder; ++m2) {
                // the product is commutative: compute it with its factors in one canonical
                // order, so that (t, m1, m2) and its mirror (t', m2, m1) get the same bits
                if (d1 > d2 || (d1 == d2 && m1 > m2)) product_dense(d2, d1, m2, m1, dense);
                else product_dense(d1, d2, m1, m2, dense);
                int kmax = m1 + m2 - d1 - d2;
                int kmin = -1;
                for (int k = (kmax >= 0 ? kmax % 2 : 0); k <= kmax; k += 2)
                    if (dense[k] != 0.0L) { kmin = k; break; }
                int cnt = 0;
                if (kmin >= 0) {
                    cnt = (kmax - kmin) / 2 + 1;
                    for (int r = 0; r < cnt; ++r) {
                        double c = (double)dense[kmin + 2 * r];
                        float hi = (float)c;
                        T.lin_coef[off + r] = c;
                        T.lin_coef_ff[2 * (off + r)] = hi;
                        T.lin_coef_ff[2 * (off + r) + 1] = (float)(c - (double)hi);
                    }
                } else {
                    kmin = 0;
                }
                T.lin_idx[lin_slot(t, m1, m2)] = (kmin & 0xff) | ((cnt & 0xff) << 8) | ((off & 0xffff) << 16);
                off += cnt;
            }
    }
    T.n_coef = off;
    return &T;
}

}  // namespace

const HostTables& host_tables() {
    static std::once_flag once;
    static HostTables* T = nullptr;
    std::call_once(once, [] { T = build(); });
    return *T;
}

}  // namespace p2s
