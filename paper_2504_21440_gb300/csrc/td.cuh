// Coefficient of a time-dependent Hamiltonian term (QobjEvo form, paper
// Sec. 2): f(t) = (amp_re + i amp_im) * env(t) * g(omega t + phi), with
// g = cos or exp(i .) and env(t) = exp(-(t - t0)^2 / (2 sigma^2)) when
// sigma > 0.  Evaluated in FP64, out of line (it runs once per term and
// stage time, and inlined its FP64 temporaries crowd the solver loops).
#pragma once

#include "internal.h"

namespace qtl {

static __device__ __noinline__ double2 td_coef(const qtl_coef& c, double t) {
    double env = 1.0;
    if (c.sigma > 0.0) {
        const double d = t - c.t0;
        env = exp(-d * d / (2.0 * c.sigma * c.sigma));
    }
    double sn, cs;
    sincos(c.omega * t + c.phi, &sn, &cs);
    const double gr = cs, gi = c.kind == QTL_COEF_EXP ? sn : 0.0;
    const double ar = c.amp_re * env, ai = c.amp_im * env;
    return make_double2(ar * gr - ai * gi, ar * gi + ai * gr);
}

}  // namespace qtl
