// Coupling factor of Eq. (2) (arXiv:1703.09619) for the metric kind, shared by the
// moment kernels and the coarse-feature kernel.
//
// geo[] holds one element's map in the form the kernels precompute:
//   geo[8 i + j]  trilinear coefficients of coordinate i: x_i = sum_j geo[8i+j] (1,u,v,w,uv,uw,vw,uvw)_j
//   geo[24 + i]   bulge vector a * b_i
//   geo[27]       eps amplitude A
//   geo[31 + j]   trilinear coefficients of the phase k . x,   geo[39] = k . (a b)
#pragma once

#include <cuda_runtime.h>

namespace p2s {

// Coupling factors of the metric kind at one point; writes K[s] for the 6 unique pairs.
// J = dx/d(u,v,w) of the trilinear-plus-bulge map; cofactors C; det = J row 0 . C row 0;
// K = eps detJ J^-1 J^-T = (eps / det) C^T C  (since J^-1 = C^T / det).
__device__ __forceinline__ bool metric_alpha(const double* geo, double u, double v, double w, double cu,
                                             double su, double cv, double sv, double cw, double sw,
                                             double* K) {
    const double hp = -1.5707963267948966;  // -pi/2
    double uv = u * v, uw = u * w, vw = v * w, uvw = uv * w;
    double beta = cu * cv * cw;
    double dbu = hp * su * cv * cw, dbv = hp * cu * sv * cw, dbw = hp * cu * cv * sw;
    double J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double* c = geo + 8 * i;
        double g = geo[24 + i];
        J[i][0] = fma(g, dbu, fma(c[7], vw, fma(c[5], w, fma(c[4], v, c[1]))));
        J[i][1] = fma(g, dbv, fma(c[7], uw, fma(c[6], w, fma(c[4], u, c[2]))));
        J[i][2] = fma(g, dbw, fma(c[7], uv, fma(c[6], v, fma(c[5], u, c[3]))));
    }
    const double* th = geo + 31;
    double theta = fma(geo[39], beta,
                       fma(th[7], uvw, fma(th[6], vw, fma(th[5], uw, fma(th[4], uv,
                           fma(th[3], w, fma(th[2], v, fma(th[1], u, th[0]))))))));
    double eps = fma(geo[27], sin(theta), 1.0);
    double C[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            C[i][j] = fma(J[i1][j1], J[i2][j2], -J[i1][j2] * J[i2][j1]);
        }
    double det = fma(J[0][0], C[0][0], fma(J[0][1], C[0][1], J[0][2] * C[0][2]));
    double sc = eps / det;
    const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        int i = pi_[s], j = pj_[s];
        K[s] = sc * fma(C[0][i], C[0][j], fma(C[1][i], C[1][j], C[2][i] * C[2][j]));
    }
    return det > 0.0;
}

}  // namespace p2s
