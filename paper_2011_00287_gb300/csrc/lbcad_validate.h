// lbcad_validate.h -- host-side checks of a grid and its parameters, shared by every entry
// point that takes an lbcad_grid and lbcad_params (lbcad_create*, lbcad_step_noalloc).
#pragma once

#include <cmath>
#include <string>

#include "lbcad.h"

namespace lbcad {

// Every floating-point parameter of Eqs. 1-11 and of the initial state is finite.
inline bool finite_params(const lbcad_params& p) {
  const double v[] = {p.tau, p.rho0, p.A0, p.chi0, p.chis, p.K, p.q0, p.gammaQ, p.xi, p.a, p.b, p.kphi,
                      p.M, p.W, p.zeta, p.R, p.centre[0], p.centre[1], p.centre[2], p.S0, p.noise};
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

// Empty when the grid and parameters are acceptable, else the reason.
inline std::string validate(const lbcad_grid& g, const lbcad_params& p) {
  if (g.nx < 4 || g.ny < 4 || g.nz < 4) return "grid: every edge must be >= 4";
  if ((long long)g.nx * g.ny * g.nz > (1LL << 31)) return "grid: more than 2^31 sites";
  if (!finite_params(p)) return "params: non-finite value";
  if (!(p.tau > 0.5)) return "params: tau must be > 1/2";
  if (!(p.rho0 > 0.0)) return "params: rho0 must be > 0";
  if (p.precision != LBCAD_FP32 && p.precision != LBCAD_FP64) return "params: precision must be FP32 or FP64";
  if (p.integrator != LBCAD_EULER && p.integrator != LBCAD_HEUN) return "params: unknown integrator";
  if (p.coupling != LBCAD_LAGGED && p.coupling != LBCAD_SYNC) return "params: unknown coupling";
  if (p.lattice != LBCAD_D3Q19 && p.lattice != LBCAD_D3Q15) return "params: unknown lattice";
  if (p.lb_form != LBCAD_LB_BODY_FORCE && p.lb_form != LBCAD_LB_STRESS_EQ) return "params: unknown lb_form";
  if (p.stencil != LBCAD_STENCIL_ISO && p.stencil != LBCAD_STENCIL_R2) return "params: unknown stencil";
  return "";
}

}  // namespace lbcad
