// The paper's control plane around the hot path (host code):
//   * ConstructMicroBatch (Alg. 1) with the latency model of Eq. 5, the
//     throughput / latency bookkeeping of Eqs. 3-4 and the targets of Eqs. 1-2;
//   * MapDevice (Alg. 2) with the per-operation costs of Eqs. 6-8;
//   * the online regression of the inflection point (Eq. 9).
// Readings where the paper is ambiguous: Eq. 2's target is the mean of the past
// MaxLat; Eq. 3 sums over all partitions; the first non-empty micro-batch is
// admitted (AvgThPut_-1 is undefined); policy GUARDED re-evaluates buffered
// data on every poll and admits when EstMaxLat + poll period reaches the
// target (policy PAPER is Alg. 1 as printed); Eq. 9 falls back to
// (mean InfPT, 0, 0) when its normal matrix is singular.
#include <algorithm>
#include <cmath>
#include <deque>
#include <vector>

#include "../../include/lmstream.h"

namespace {

struct Ds {
  double arrival_ms;
  double bytes;
};

}  // namespace

struct lms_admission {
  double slide_ms = 0.0;
  int policy = LMS_ADMIT_PAPER;
  double poll_ms = 10.0;
  std::vector<Ds> buffered;
  std::vector<Ds> admitted;
  double admitted_at = 0.0;
  double sum_bytes = 0.0;    // Eq. 3 numerator over past micro-batches
  double sum_proc = 0.0;     // Eq. 3 denominator
  double sum_maxlat = 0.0;   // Eq. 2 target: mean of past MaxLat
  long long batches = 0;
  double last_est = 0.0;
  lms_proc_predictor pred = nullptr;
  void* pred_ctx = nullptr;
};

struct lms_regressor {
  int history = 0;
  std::deque<double> thp, lat, inf;
};

extern "C" {

lms_admission* lms_admission_create(double slide_ms, int32_t policy, double poll_ms) {
  if (slide_ms < 0 || (policy != LMS_ADMIT_PAPER && policy != LMS_ADMIT_GUARDED) || poll_ms < 0)
    return nullptr;
  lms_admission* a = new lms_admission();
  a->slide_ms = slide_ms;
  a->policy = policy;
  a->poll_ms = poll_ms;
  return a;
}

void lms_admission_destroy(lms_admission* a) { delete a; }

void lms_admission_set_predictor(lms_admission* a, lms_proc_predictor fn, void* ctx) {
  if (!a) return;
  a->pred = fn;
  a->pred_ctx = ctx;
}

int32_t lms_admission_poll(lms_admission* a, double now_ms, const double* arrival_ms,
                           const double* bytes, int32_t n_new, double* est_ms,
                           int32_t* n_admitted) {
  if (!a || n_new < 0 || (n_new > 0 && (!arrival_ms || !bytes))) return LMS_EINVAL;
  if (n_new == 0 && (a->policy == LMS_ADMIT_PAPER || a->buffered.empty())) {
    if (n_admitted) *n_admitted = 0;
    return 0;
  }
  // tmp = buffered U new, new sorted by creation (arrival) time
  std::vector<Ds> fresh(n_new);
  for (int i = 0; i < n_new; ++i) fresh[i] = {arrival_ms[i], bytes[i]};
  std::stable_sort(fresh.begin(), fresh.end(),
                   [](const Ds& x, const Ds& y) { return x.arrival_ms < y.arrival_ms; });
  std::vector<Ds> tmp = a->buffered;
  tmp.insert(tmp.end(), fresh.begin(), fresh.end());
  double max_buff = 0.0, total = 0.0;
  for (size_t j = 0; j < tmp.size(); ++j) {
    max_buff = j == 0 ? now_ms - tmp[j].arrival_ms : std::max(max_buff, now_ms - tmp[j].arrival_ms);
    total += tmp[j].bytes;
  }
  bool admit;
  if (a->batches == 0) {
    admit = true;  // AvgThPut_-1 is undefined: the first non-empty batch goes
    a->last_est = max_buff;
  } else {
    // Eq. 5 (or an installed predictor of the processing time)
    const double proc = a->pred ? a->pred(a->pred_ctx, total, (int32_t)tmp.size())
                                : total / (a->sum_bytes / a->sum_proc);
    const double est = max_buff + proc;
    a->last_est = est;
    const double target = a->slide_ms > 0 ? a->slide_ms : a->sum_maxlat / (double)a->batches;
    admit = a->policy == LMS_ADMIT_GUARDED ? est + a->poll_ms >= target : est >= target;
  }
  if (est_ms) *est_ms = a->last_est;
  if (admit) {
    a->admitted = std::move(tmp);
    a->admitted_at = now_ms;
    a->buffered.clear();
    if (n_admitted) *n_admitted = (int32_t)a->admitted.size();
    return 1;
  }
  a->buffered = std::move(tmp);
  if (n_admitted) *n_admitted = 0;
  return 0;
}

double lms_admission_complete(lms_admission* a, double proc_ms) {
  if (!a || a->admitted.empty()) return -1.0;
  double max_buff = 0.0, total = 0.0;
  for (size_t j = 0; j < a->admitted.size(); ++j) {
    const double b = a->admitted_at - a->admitted[j].arrival_ms;
    max_buff = j == 0 ? b : std::max(max_buff, b);
    total += a->admitted[j].bytes;
  }
  const double maxlat = max_buff + proc_ms;  // Eq. 4
  a->sum_bytes += total;                     // Eq. 3
  a->sum_proc += proc_ms;
  a->sum_maxlat += maxlat;
  a->batches += 1;
  a->admitted.clear();
  return maxlat;
}

double lms_admission_avg_thput(const lms_admission* a) {
  return (a && a->sum_proc > 0) ? a->sum_bytes / a->sum_proc : 0.0;
}

int32_t lms_admission_buffered(const lms_admission* a) {
  return a ? (int32_t)a->buffered.size() : 0;
}

double lms_admission_last_estimate(const lms_admission* a) { return a ? a->last_est : 0.0; }

lms_status lms_map_device(const int32_t* ops, int32_t n_ops, double batch_bytes, int32_t num_cores,
                          double infpt_bytes, double base_trans_cost, int32_t* device,
                          double* cpu_cost, double* gpu_cost) {
  // Table II base costs, in LMS_QOP_* order
  static const double kBase[8] = {1.0, 1.0, 1.0, 0.9, 0.9, 0.9, 0.8, 0.8};
  if (!ops || n_ops <= 0 || num_cores <= 0 || !(batch_bytes > 0) || !(infpt_bytes > 0) || !device)
    return LMS_EINVAL;
  for (int o = 0; o < n_ops; ++o)
    if (ops[o] < 0 || ops[o] > 7) return LMS_EINVAL;
  const double part = batch_bytes / num_cores;
  for (int o = 0; o < n_ops; ++o) {
    const double b = kBase[ops[o]];
    double cpu = b * part / infpt_bytes;                  // Eq. 6
    double gpu = b * infpt_bytes / part;                  // Eq. 7
    const double trans = base_trans_cost * part / infpt_bytes;  // Eq. 8
    if (o == 0 || o == n_ops - 1 || device[o - 1] == 1) gpu += trans;
    else cpu += trans;
    device[o] = gpu > cpu ? 1 : 0;
    if (cpu_cost) cpu_cost[o] = cpu;
    if (gpu_cost) gpu_cost[o] = gpu;
  }
  return LMS_OK;
}

lms_regressor* lms_regressor_create(int32_t history_len) {
  if (history_len < 0) return nullptr;
  lms_regressor* r = new lms_regressor();
  r->history = history_len;
  return r;
}

void lms_regressor_destroy(lms_regressor* r) { delete r; }

void lms_regressor_add(lms_regressor* r, double thput, double lat, double infpt) {
  if (!r) return;
  r->thp.push_back(thput);
  r->lat.push_back(lat);
  r->inf.push_back(infpt);
  if (r->history > 0 && (int)r->thp.size() > r->history) {
    r->thp.pop_front();
    r->lat.pop_front();
    r->inf.pop_front();
  }
}

namespace {
// Eigenvalues of a symmetric 3x3 matrix (closed form, trigonometric method).
void sym3_eigen(const double A[3][3], double ev[3]) {
  const double p1 = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
  const double q = (A[0][0] + A[1][1] + A[2][2]) / 3.0;
  if (p1 == 0.0) {
    ev[0] = A[0][0];
    ev[1] = A[1][1];
    ev[2] = A[2][2];
    return;
  }
  const double p2 = (A[0][0] - q) * (A[0][0] - q) + (A[1][1] - q) * (A[1][1] - q) +
                    (A[2][2] - q) * (A[2][2] - q) + 2.0 * p1;
  const double p = std::sqrt(p2 / 6.0);
  double B[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[i][j] = (A[i][j] - (i == j ? q : 0.0)) / p;
  const double detB = B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
                      B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                      B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
  double r = detB / 2.0;
  r = std::max(-1.0, std::min(1.0, r));
  const double phi = std::acos(r) / 3.0;
  const double kPi = 3.14159265358979323846;
  ev[0] = q + 2.0 * p * std::cos(phi);
  ev[2] = q + 2.0 * p * std::cos(phi + 2.0 * kPi / 3.0);
  ev[1] = 3.0 * q - ev[0] - ev[2];
}
}  // namespace

lms_status lms_regressor_fit(lms_regressor* r, double target_thput, double target_lat,
                             double* beta, double* infpt) {
  if (!r || !beta || !infpt) return LMS_EINVAL;
  const size_t n = r->thp.size();
  double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0}, mean = 0.0;
  for (size_t k = 0; k < n; ++k) {
    const double x[3] = {1.0, r->thp[k], r->lat[k]};
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) A[i][j] += x[i] * x[j];
      b[i] += x[i] * r->inf[k];
    }
    mean += r->inf[k];
  }
  bool singular = n < 3;
  if (!singular) {
    double ev[3];
    sym3_eigen(A, ev);
    const double hi = std::max(std::fabs(ev[0]), std::max(std::fabs(ev[1]), std::fabs(ev[2])));
    const double lo = std::min(std::fabs(ev[0]), std::min(std::fabs(ev[1]), std::fabs(ev[2])));
    singular = !(lo > 0.0) || hi / lo > 1e14;
  }
  if (singular) {
    beta[0] = n ? mean / (double)n : 150.0 * 1024.0;
    beta[1] = 0.0;
    beta[2] = 0.0;
  } else {
    // Gaussian elimination with partial pivoting on the normal equations
    double M[3][4];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
      M[i][3] = b[i];
    }
    for (int c = 0; c < 3; ++c) {
      int piv = c;
      for (int i = c + 1; i < 3; ++i)
        if (std::fabs(M[i][c]) > std::fabs(M[piv][c])) piv = i;
      for (int j = 0; j < 4; ++j) std::swap(M[c][j], M[piv][j]);
      for (int i = c + 1; i < 3; ++i) {
        const double f = M[i][c] / M[c][c];
        for (int j = c; j < 4; ++j) M[i][j] -= f * M[c][j];
      }
    }
    for (int i = 2; i >= 0; --i) {
      double s = M[i][3];
      for (int j = i + 1; j < 3; ++j) s -= M[i][j] * beta[j];
      beta[i] = s / M[i][i];
    }
  }
  *infpt = beta[0] + beta[1] * target_thput + beta[2] * target_lat;
  return n < 3 ? LMS_EAGAIN : LMS_OK;
}

}  // extern "C"
