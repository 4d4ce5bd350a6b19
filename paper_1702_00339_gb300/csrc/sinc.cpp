// Default R-term Gaussian-sum rule for 1/z (Sec. 2.2, Eqs. 2.6-2.7).
// Reading (the paper prints no nodes): t = e^u in
//   1/z = (2/sqrt(pi)) int exp(u - z^2 e^{2u}) du,
// R-1 trapezoid nodes on [u_lo, u_hi] with half end weights plus one tail
// node for (-inf, u_lo) (weight (2/sqrt(pi)) e^{u_lo}, t = e^{u_lo}/sqrt 3),
// (u_lo, u_hi) chosen by a fixed coarse-to-fine search minimising the
// maximum relative error on 301 log-spaced points of [1, zmax/zmin].
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/fock.h"

namespace {

const double kTwoOverSqrtPi = 1.1283791670955125739;

void rule(int R, double ulo, double uhi, std::vector<double>& t, std::vector<double>& c) {
  int n = R - 1;
  double hs = (uhi - ulo) / (n - 1);
  t.assign(R, 0.0);
  c.assign(R, 0.0);
  t[0] = std::exp(ulo) / std::sqrt(3.0);
  c[0] = kTwoOverSqrtPi * std::exp(ulo);
  for (int q = 0; q < n; ++q) {
    double u = ulo + hs * q;
    t[q + 1] = std::exp(u);
    c[q + 1] = kTwoOverSqrtPi * hs * std::exp(u) * ((q == 0 || q == n - 1) ? 0.5 : 1.0);
  }
}

double max_rel_err(const std::vector<double>& t, const std::vector<double>& c, double rho) {
  const int nz = 301;
  double lr = std::log(rho), e = 0.0;
  for (int i = 0; i < nz; ++i) {
    double z = std::exp(lr * i / (nz - 1));
    double s = 0.0;
    for (size_t q = 0; q < t.size(); ++q) s += c[q] * std::exp(-(z * t[q]) * (z * t[q]));
    e = std::fmax(e, std::fabs(s * z - 1.0));
  }
  return e;
}

std::mutex g_mu;
std::map<std::tuple<int, double, double>, std::tuple<std::vector<double>, std::vector<double>, double>> g_cache;

}  // namespace

extern "C" int fock_sinc_table(int R, double zmin, double zmax, double* t, double* c, double* err) {
  if (R < 3 || R > 64 || !(zmin > 0.0) || !(zmax > zmin) || !t || !c) return FOCK_EINVAL;
  auto key = std::make_tuple(R, zmin, zmax);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      for (int q = 0; q < R; ++q) { t[q] = std::get<0>(it->second)[q]; c[q] = std::get<1>(it->second)[q]; }
      if (err) *err = std::get<2>(it->second);
      return FOCK_OK;
    }
  }
  const double rho = zmax / zmin;
  std::vector<double> tt, cc;
  double best = 1e300, blo = -15.0, bhi = 1.0;
  const double steps_lo[3] = {1.0, 0.2, 0.04}, steps_hi[3] = {0.25, 0.05, 0.01};
  for (int level = 0; level < 3; ++level) {
    std::vector<double> los, his;
    if (level == 0) {
      for (int i = 0;; ++i) { double v = -30.0 + i * steps_lo[0]; if (v > -1.99) break; los.push_back(v); }
      for (int i = 0;; ++i) { double v = 0.0 + i * steps_hi[0]; if (v > 3.001) break; his.push_back(v); }
    } else {
      for (int i = -5; i <= 5; ++i) los.push_back(blo + steps_lo[level] * i);
      for (int i = -5; i <= 5; ++i) his.push_back(bhi + steps_hi[level] * i);
    }
    double clo = blo, chi = bhi;
    for (double ulo : los)
      for (double uhi : his) {
        if (uhi <= ulo) continue;
        rule(R, ulo, uhi, tt, cc);
        double e = max_rel_err(tt, cc, rho);
        if (e < best) { best = e; clo = ulo; chi = uhi; }
      }
    blo = clo;
    bhi = chi;
  }
  rule(R, blo, bhi, tt, cc);
  for (int q = 0; q < R; ++q) { tt[q] /= zmin; cc[q] /= zmin; }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = std::make_tuple(tt, cc, best);
  }
  for (int q = 0; q < R; ++q) { t[q] = tt[q]; c[q] = cc[q]; }
  if (err) *err = best;
  return FOCK_OK;
}

extern "C" int fock_default_range(const fock_problem* p, double* zmin, double* zmax) {
  if (!p || p->n0 <= 0 || !(p->b0 > 0.0)) return FOCK_EINVAL;
  double h = p->b0 / p->n0, ext = 0.0;
  for (int a = 0; a < 3; ++a) {
    double e = p->N[a] * h + (p->L[a] / 2 + 1) * p->b0;
    ext += e * e;
  }
  if (zmin) *zmin = h * 1e-2;
  if (zmax) *zmax = 2.0 * std::sqrt(ext);
  return FOCK_OK;
}
