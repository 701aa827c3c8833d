// Bulk-surface coupling terms at one surface point (Sections 5.5 and 5.6), shared by the
// coupling kernels and the host-side evaluation sexpe_coupling_terms.
#pragma once

#include "internal.h"

namespace sexpe {

// The coupling terms at one surface point from the bulk values (ub, vb) on the
// boundary and the surface values (r, s): add[0], add[1] go to the bulk F of the
// boundary node, add[2], add[3] to the surface F (Sections 5.5 and 5.6).
__host__ __device__ inline void couple_terms(const CoupleArgs& a, double ub, double vb, double r, double s,
                                             double* add) {
    if (a.kind == 0) {      // Robin exchange of eqs. bulkball
        const double ju = a.z[0] * (a.z[1] * r - a.z[2] * ub), jv = a.z[0] * (a.e[0] * s - a.e[1] * vb);
        add[0] = a.d0 * a.coef * ju;                 // d_u grad u . n
        add[1] = a.coef * jv;                        // delta grad v . n
        add[2] = -ju;
        add[3] = -jv;
    } else {                // DIB kinetics of eqs. bulkcylnl, bulk lifted by the top values
        const double u = ub + a.u_top, v = vb + a.v_top;
        const double P = a.z[1] * u * (1.0 - s) * r - a.z[2] * r * r * r - a.z[3] * (s - a.z[4]);
        const double Q = a.e[0] * v * (1.0 + a.e[1] * r) * (1.0 - s) * (1.0 - a.e[2] * (1.0 - s)) -
                         a.e[3] * (1.0 + a.e[4] * r) * s * (1.0 + a.e[2] * s);
        const double gu = -a.z[0] * a.a3 * P, gv = -a.z[0] * a.b3 * Q;    // grad . n on z = 0
        add[0] = a.d0 * a.coef * gu;
        add[1] = a.d1 * a.coef * gv;
        add[2] = a.z[0] * P;
        add[3] = a.z[0] * Q;
    }
}

}  // namespace sexpe
