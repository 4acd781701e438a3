// gfdtd_medium.h -- host-side construction of an instance's device record
// (InstDev) and profile tables from its moving medium.  Shared by the context
// path (gfdtd_api.cu) and the allocation-free entry point (gfdtd_noalloc.cu),
// so both hand the kernels identical records.
#pragma once

#include "gfdtd_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gfdtd {

// A position in cells as 32.32 fixed point (units of 2^-32 cell).
inline long long to_fixed(double x) { return llround(ldexp(x, 32)); }

// Star-relation coefficients of a uniform medium (kind 0: moving perturbation,
// Eq. const_1d: E* = D/eps - beta B, H* = B/mu - beta D; kind 1: moving matter,
// Eq. const_3d with the footnote tensors of Eq. const_3d_regular solved for
// E*, H*): E* = ie D - bc B, H* = im B - bc D.
inline void medium_coefs(int kind, double beta, double e, double m, double* ie, double* im, double* bc) {
  if (kind == 0) {
    *ie = 1.0 / e;
    *im = 1.0 / m;
    *bc = beta;
    return;
  }
  const double den = e * m - beta * beta, g = 1.0 - beta * beta;
  *ie = g * m / den;
  *im = g * e / den;
  *bc = beta * g / den;
}

// The FP32 kernels' coupling weight cb = S beta_c / 2, rounded to a multiple of
// 2^-24.  With c = 2 |cb| and a = 1 - c (moving perturbation: c = |beta| S
// exactly as in the scheme), every weight the FP32 updates use and every sum
// of them (a + c, a +- cb, c -+ cb) is then exact in FP32, so the discrete
// identities of Table 1 that the scheme relies on -- the upwind weights a + c
// add to one, and the upwind difference and the Ba/Bb average cancel on a
// uniform field when c = 2 |cb| -- hold exactly.  Rounded independently to
// FP32, the three weights miss those identities by a few units of 2^-25 and
// the fields drift by a multiple of that per step (about 2e-4 relative after
// 8000 steps; with this rounding the drift is gone and only unbiased
// per-operation rounding remains).
inline float fp32_coupling(double cb) {
  return (float)(std::nearbyint(std::ldexp(cb, 24)) * std::ldexp(1.0, -24));
}

// One instance's moving medium, as gfdtd_set_medium receives it.
struct MediumSpec {
  int kind = 0;              // 0 moving perturbation, 1 moving matter
  double beta = 0.0;
  int interp = 0;            // 0 LAYERS, 1 LINEAR
  int n = 1;                 // values (layers or knots)
  const double* z = nullptr; // n - 1 boundaries (LAYERS) or n knots (LINEAR)
  const double* eps = nullptr;
  const double* mu = nullptr;
  long long absorb_width = 0;
  double absorb_sigma = 0.0;
};

// Fills the medium part of `d` (every field but off, nz, nz_pad, src0, nsrc,
// prb0, nprb, tf0, ntf) and appends the instance's entries to the profile
// tables (zq is padded to the tables' length).
inline void fill_instance(const MediumSpec& m, double S, InstDev& d, std::vector<long long>& zq,
                          std::vector<double2>& tabE, std::vector<double2>& tabH, std::vector<float2>& tabE32,
                          std::vector<float2>& tabH32) {
  d.dq = llround(ldexp(m.beta * S, 31));
  d.n = m.n;
  d.minw = 0;
  d.tab = (int)tabE.size();
  d.a = 1.0 - std::fabs(m.beta) * S;
  d.c = std::fabs(m.beta) * S;
  d.S = S;
  d.inv_S = 1.0 / S;
  d.beta = m.beta;
  d.cb = 0.5 * S * m.beta;
  d.cb32 = fp32_coupling(d.cb);
  d.c32 = 2.0f * std::fabs(d.cb32);
  d.a32 = 1.0f - d.c32;
  d.sm32 = 0.0f;
  d.abs_w = (int)m.absorb_width;
  d.abs_sigma = m.absorb_sigma;
  int flags = 0;
  if (m.beta >= 0.0) flags |= F_POS;
  if (m.kind == 1) flags |= F_MATTER;
  const int n = m.n;
  if (m.interp == 1) {
    flags |= F_LINEAR;
    // a moving-perturbation profile whose eps (or mu) knots are all equal has a
    // uniform S/eps (or S/mu): the kernels then skip that side's interpolation
    bool econst = m.kind != 1, mconst = m.kind != 1;
    for (int k = 0; k < n; ++k) {
      zq.push_back(to_fixed(m.z[k]));
      const double2 v = make_double2(m.eps[k], m.mu[k]);
      tabE.push_back(v);
      tabH.push_back(v);
      tabE32.push_back(make_float2((float)v.x, (float)v.y));
      tabH32.push_back(make_float2((float)v.x, (float)v.y));
      if (m.eps[k] != m.eps[0]) econst = false;
      if (m.mu[k] != m.mu[0]) mconst = false;
    }
    if (econst) flags |= F_EPS_CONST;
    if (mconst) flags |= F_MU_CONST;
    d.sm32 = (float)(S / m.mu[0]);
  } else {
    bool econst = true, mconst = true;
    for (int k = 0; k < n; ++k) {
      if (k < n - 1) zq.push_back(to_fixed(m.z[k]));
      double ie, im, bc;
      medium_coefs(m.kind, m.beta, m.eps[k], m.mu[k], &ie, &im, &bc);
      const double2 e = make_double2(S * ie, 0.5 * S * bc);
      const double2 h = make_double2(S * im, 0.5 * S * bc);
      if (k > 0 && (e.x != tabE[d.tab].x || e.y != tabE[d.tab].y)) econst = false;
      if (k > 0 && (h.x != tabH[d.tab].x || h.y != tabH[d.tab].y)) mconst = false;
      tabE.push_back(e);
      tabH.push_back(h);
      tabE32.push_back(make_float2((float)e.x, fp32_coupling(e.y)));
      tabH32.push_back(make_float2((float)h.x, fp32_coupling(h.y)));
    }
    // boundaries move rigidly, so their node indices stay at least floor(width) - 1 apart
    double wmin = 1e30;
    for (int k = 1; k + 1 < n; ++k) wmin = std::min(wmin, m.z[k] - m.z[k - 1]);
    d.minw = wmin > 1e9 ? (1 << 30) : std::max(0, (int)std::floor(wmin) - 1);
    if (econst) flags |= F_EPS_CONST;
    if (mconst) flags |= F_MU_CONST;
    d.sm32 = (float)tabH[d.tab].x;
  }
  while (zq.size() < tabE.size()) zq.push_back(0);   // keep zq aligned with the tables
  d.flags = flags;
}

}  // namespace gfdtd
