// Scalar recurrences of preconditioned MINRES (Paige & Saunders 1975), shared
// by the single-mesh and the batched kernels: the Lanczos start and, per
// iteration, beta_{k+1}, the Givens rotation of the tridiagonal QR
// factorisation, the solution-update coefficients and the stop test
// phibar <= rtol * beta1.
#pragma once

#include <climits>
#include <cmath>

#include "tmop_internal.h"

namespace tmop {

__device__ __forceinline__ void minres_start_scalars(MinresState *st, double bb)
{
    const double b1 = sqrt(fmax(bb, 0.0));
    st->beta1 = b1;
    st->beta = b1;
    st->beta_old = 0.0;
    st->alpha = 0.0;
    st->dbar = 0.0;
    st->eps = 0.0;
    st->eps_old = 0.0;
    st->phibar = b1;
    st->cs = -1.0;
    st->sn = 0.0;
    st->gamma = 1.0;
    st->delta = 0.0;
    st->phi = 0.0;
    st->stop_iter = (b1 > 0.0) ? INT_MAX : 0;
    st->breakdown = 0;
    st->iters = 0;
    st->k = 0;
}

// bb = (r_{k+1}, M^-1 r_{k+1}) of iteration k.
__device__ __forceinline__ void minres_beta_scalars(MinresState *st, double bb, int k, double rtol,
                                                    int fixed_its)
{
    st->iters = k;
    if (!(bb >= 0.0)) {              // negative (M^-1 not positive) or not finite
        st->breakdown = 1;
        st->stop_iter = k - 1;       // discard this iteration
        return;
    }
    st->beta_old = st->beta;
    const double beta = sqrt(bb);
    st->beta = beta;
    const double alpha = st->alpha;
    st->eps_old = st->eps;
    const double delta = st->cs * st->dbar + st->sn * alpha;
    const double gbar = st->sn * st->dbar - st->cs * alpha;
    st->eps = st->sn * beta;
    st->dbar = -st->cs * beta;
    double gamma = sqrt(gbar * gbar + beta * beta);
    if (gamma < 1e-300) gamma = 1e-300;
    st->gamma = gamma;
    st->delta = delta;
    st->cs = gbar / gamma;
    st->sn = beta / gamma;
    st->phi = st->cs * st->phibar;
    st->phibar = st->sn * st->phibar;
    if ((!fixed_its && st->phibar <= rtol * st->beta1) || beta == 0.0) st->stop_iter = k;
}

}  // namespace tmop
