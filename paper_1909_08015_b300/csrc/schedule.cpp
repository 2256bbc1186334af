// Sampling probabilities of the paper's integration controller (Sec. IV.C):
// the time to process N samples is N sum_j p_j t_j and the variance of the
// total (1/N) sum_j C_j^2 / p_j, C_j = sigma_j sqrt(N_j); their product is
// smallest at p_j proportional to C_j / sqrt(t_j).
#include <cmath>
#include <cstdint>

#include "../../include/ae.h"

extern "C" int ae_schedule_probabilities(const double *sigma, const uint64_t *N, const double *t, int n,
                                         double p_floor, double *p) {
  if (!sigma || !N || !t || !p || n <= 0 || !(p_floor >= 0) || p_floor > 1) return AE_ERR_ARG;
  double sum = 0;
  for (int j = 0; j < n; ++j) {
    double w = 0;
    if (t[j] > 0 && std::isfinite(sigma[j]) && sigma[j] > 0)
      w = sigma[j] * std::sqrt((double)N[j]) / std::sqrt(t[j]);
    if (!std::isfinite(w) || w < 0) w = 0;
    p[j] = w;
    sum += w;
  }
  if (!(sum > 0)) {
    for (int j = 0; j < n; ++j) p[j] = 1.0 / n;
    return AE_OK;
  }
  const double lo = p_floor / n;
  double tot = 0;
  for (int j = 0; j < n; ++j) {
    p[j] = p[j] / sum;
    if (p[j] < lo) p[j] = lo;
    tot += p[j];
  }
  for (int j = 0; j < n; ++j) p[j] /= tot;
  return AE_OK;
}

// Two independent calculations combined as in Sec. V: graph by graph by
// inverse-variance weighting, then summed with Eq. eq_sigma_sum.
extern "C" int ae_combine_runs(const double *v1, const double *s1, const double *v2, const double *s2, int n,
                               double *v_out, double *s_out, double *total, double *total_sigma) {
  if (!v1 || !s1 || !v2 || !s2 || n <= 0) return AE_ERR_ARG;
  double tot = 0, var = 0;
  for (int j = 0; j < n; ++j) {
    double v, s;
    if (s1[j] > 0 && s2[j] > 0) {
      const double w1 = 1.0 / (s1[j] * s1[j]), w2 = 1.0 / (s2[j] * s2[j]);
      v = (w1 * v1[j] + w2 * v2[j]) / (w1 + w2);
      s = std::sqrt(1.0 / (w1 + w2));
    } else if (s1[j] > 0 || s2[j] > 0) {   // one exact value: it decides
      v = s1[j] > 0 ? v2[j] : v1[j];
      s = 0.0;
    } else {
      v = 0.5 * (v1[j] + v2[j]);
      s = 0.0;
    }
    if (v_out) v_out[j] = v;
    if (s_out) s_out[j] = s;
    tot += v;
    var += s * s;
  }
  if (total) *total = tot;
  if (total_sigma) *total_sigma = std::sqrt(var);
  return AE_OK;
}

// Widths of the paper's acceptance test (Sec. IV.A, Eq. eq_interval_accept):
// width_j = (1/4) sigma_j sqrt(sum_l sigma_l^2) / sum_l sigma_l.  Summed
// over the graphs the widths give (1/4) sqrt(sum_l sigma_l^2): the round-off
// error of the set stays below a quarter of its sigma_down.
extern "C" int ae_accept_widths(const double *sigma, int n, double *width) {
  if (!sigma || !width || n <= 0) return AE_ERR_ARG;
  double s1 = 0, s2 = 0;
  for (int j = 0; j < n; ++j)
    if (std::isfinite(sigma[j]) && sigma[j] > 0) { s1 += sigma[j]; s2 += sigma[j] * sigma[j]; }
  for (int j = 0; j < n; ++j)
    width[j] = (s1 > 0 && std::isfinite(sigma[j]) && sigma[j] > 0) ? 0.25 * sigma[j] * std::sqrt(s2) / s1 : 0.0;
  return AE_OK;
}
