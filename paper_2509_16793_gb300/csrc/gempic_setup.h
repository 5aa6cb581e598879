// Host-side checks and physics parameters shared by gempic_create and gempic_step_noalloc:
// species, density channel, stability bound and the FP32 fixed-point range.
#pragma once
#include <algorithm>
#include <cmath>

#include "../../include/gempic.h"
#include "gempic_internal.h"

namespace gempic {

// Fills the species and channel fields of p (qm, Qf, wd, m_over_q, ppc, poff, nlayer,
// ppc_sum, nspecies, chan_a, chan_ir2, jref) from cfg.  GEMPIC_EINVAL for a bad species or
// channel; GEMPIC_EUNSTABLE when Delta h omega_p^2 > 4 at the densest point of the profile
// (Sec. 4.2).
inline gempic_status setup_species(const gempic_config* cfg, Params& p) {
  const gempic_grid& g = cfg->grid;
  if (cfg->nspecies < 0 || cfg->nspecies > kMaxSpecies) return GEMPIC_EINVAL;
  if (cfg->nspecies > 0 && !cfg->species) return GEMPIC_EINVAL;
  // density profile factor f(r) = 1 + a exp(-r^2/R^2), a = n1/n0 - 1 (Eq. n_plasma)
  double a = 0.0, ir2 = 0.0;
  if (cfg->channel) {
    const gempic_channel& ch = *cfg->channel;
    if (!(ch.n1_over_n0 >= 0) || !(ch.radius > 0) || !std::isfinite(ch.n1_over_n0) ||
        !std::isfinite(ch.radius))
      return GEMPIC_EINVAL;
    a = ch.n1_over_n0 - 1.0;
    ir2 = 1.0 / (ch.radius * ch.radius);
  }
  const double fmax = std::max(1.0, 1.0 + a);   // f is largest on the axis or far from it
  // zeta-step: the largest slab bounds stability, the smallest sets the fixed-point range
  double hmax = g.h, hmin = g.h;
  if (cfg->hz) {
    hmax = 0.0;
    hmin = INFINITY;
    for (int n = 0; n < g.nzeta; ++n) {
      if (!(cfg->hz[n] > 0) || !std::isfinite(cfg->hz[n])) return GEMPIC_EINVAL;
      hmax = std::max(hmax, cfg->hz[n]);
      hmin = std::min(hmin, cfg->hz[n]);
    }
  }
  double wp2 = 0.0, wmax = 0.0, qn = 0.0;
  int ppc_sum = 0, off = 0;
  for (int i = 0; i < cfg->nspecies; ++i) {
    const gempic_species& sp = cfg->species[i];
    if (sp.ppc < 1 || !(sp.mass > 0) || !(sp.density >= 0)) return GEMPIC_EINVAL;
    if (sp.density > 0 && sp.charge == 0) return GEMPIC_EINVAL;
    wp2 += sp.charge * sp.charge * sp.density / sp.mass;
    qn += sp.charge * sp.density;
    wmax = std::max(wmax, std::fabs(sp.charge * sp.density / sp.ppc));
    ppc_sum += sp.ppc;
    p.qm[i] = sp.charge / sp.mass;
    p.Qf[i] = sp.charge * sp.density * g.hx * g.hy * cfg->delta / sp.ppc;
    p.wd[i] = p.Qf[i] / (g.hx * g.hy * cfg->delta);
    p.m_over_q[i] = sp.charge != 0 ? sp.mass / sp.charge : 0.0;
    p.ppc[i] = sp.ppc;
    p.poff[i] = off;
    off += g.nx * g.ny * sp.ppc;
  }
  if (cfg->delta * hmax * wp2 * fmax > 4.0 * (1.0 + 1e-12)) return GEMPIC_EUNSTABLE;
  p.nspecies = cfg->nspecies;
  p.bg_qn = -qn;
  p.nlayer = off;
  p.ppc_sum = ppc_sum;
  p.chan_a = a;
  p.chan_ir2 = ir2;
  // fixed-point range of the FP32 deposit: 4 x the largest (rho - j_z) weight times the
  // largest transverse cell-to-slice ratio; a larger contribution takes the float path
  const double ratio = std::max(1.0, std::max(g.hx, g.hy) / hmin);
  p.jref = wmax > 0 ? 4.0 * wmax * fmax * ratio : 1.0;
  return GEMPIC_OK;
}

}  // namespace gempic
