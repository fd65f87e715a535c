// Coupling factor of Eq. (2) (arXiv:1703.09619), metric kind, in double-word arithmetic:
// shared by the double-word moment kernel and the coarse-feature kernel.
//
// geo[] holds one element's constants as double words, in the layout of alpha.cuh (trilinear
// coefficients 0..23, bulge vector 24..26, eps amplitude 27, phase coefficients 31..38, the
// bulge's phase 39).  The Jacobian at (u, v, w) is formed from constants of the point's row
// (fixed v, w) and plane (fixed w):
//   row[i] = B_i, row[3 + i] = F_i, row[6 + i] = H_i, row[9] = T0, row[10] = T1,
//   row[11] = cos(pi v/2) cos(pi w/2), row[12] = d/dv of it, row[13] = d/dw of it;
//   plane[i] = D_i, plane[3 + i] = E_i;
// so that J_iu = B_i + g_i dbeta/du, J_iv = D_i + u E_i + g_i dbeta/dv,
// J_iw = F_i + u H_i + g_i dbeta/dw and k.x = T0 + u T1 + kappa beta.
#pragma once

#include "dw.cuh"

namespace p2s {

// alpha (metric kind) at one point from the row/plane constants; returns detJ > 0.  Every
// operation is a _fast or _lazy one (dw.cuh): the error of each factor is O(u^2) against the
// scale of its operands, which the normwise error of the element matrices tolerates.  The
// Jacobian, cofactor, determinant, Gram, phase and eps sums skip the renormalisation of
// their result (_lazy): every later operation takes both words of an operand.
__device__ __forceinline__ bool metric_alpha_dw(const dw* geo, const dw* row, const dw* plane, dw u, dw Ca,
                                                dw Sa, dw* K) {
    const dw beta = dw_mul_fast(Ca, row[11]);
    const dw dbu = dw_mul_fast(Sa, row[11]);
    const dw dbv = dw_mul_fast(Ca, row[12]);
    const dw dbw = dw_mul_fast(Ca, row[13]);
    dw J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const dw g = geo[24 + i];
        J[i][0] = dw_fma_lazy(g, dbu, row[i]);
        J[i][1] = dw_fma_lazy(g, dbv, dw_fma_lazy(u, plane[3 + i], plane[i]));
        J[i][2] = dw_fma_lazy(g, dbw, dw_fma_lazy(u, row[6 + i], row[3 + i]));
    }
    const dw theta = dw_fma_lazy(geo[39], beta, dw_fma_lazy(u, row[10], row[9]));
    const dw eps = dw_add_f_lazy(dw_mul_fast(geo[27], dw_sin(theta)), 1.f);
    dw C[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            C[i][j] = dw_sub_lazy(dw_mul_fast(J[i1][j1], J[i2][j2]), dw_mul_fast(J[i1][j2], J[i2][j1]));
        }
    const dw det = dw_add_lazy(dw_mul_fast(J[0][0], C[0][0]),
                               dw_add_lazy(dw_mul_fast(J[0][1], C[0][1]), dw_mul_fast(J[0][2], C[0][2])));
    const dw sc = dw_div_fast(eps, det);
    const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int i = pi_[s], j = pj_[s];
        const dw g = dw_add_lazy(dw_mul_fast(C[0][i], C[0][j]),
                                 dw_add_lazy(dw_mul_fast(C[1][i], C[1][j]), dw_mul_fast(C[2][i], C[2][j])));
        K[s] = dw_mul_fast(sc, g);
    }
    return det.hi + det.lo > 0.f;
}

}  // namespace p2s
