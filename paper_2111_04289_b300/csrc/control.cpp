// The paper's control plane around the hot path (host code):
//   * ConstructMicroBatch (Alg. 1) with the latency model of Eq. 5, the
//     throughput / latency bookkeeping of Eqs. 3-4 and the targets of Eqs. 1-2;
//   * MapDevice (Alg. 2) with the per-operation costs of Eqs. 6-8;
//   * the online regression of the inflection point (Eq. 9).
// Readings where the paper is ambiguous: Eq. 2's target is the mean of the past
// MaxLat; Eq. 3 sums over all partitions; the first non-empty micro-batch is
// admitted (AvgThPut_-1 is undefined); policy GUARDED re-evaluates buffered
// data on every poll and admits when EstMaxLat + poll period reaches the
// target (policy PAPER is Alg. 1 as printed); Eq. 9 is solved on centred
// inputs and falls back to (mean InfPT, 0, 0) with fewer than 3 samples, a
// constant input, or collinear inputs (1 - r^2 below 1e-12).
//
// The engine runs every operation on the GPU, so Alg. 2's CPU/GPU choice is
// re-read as the choice between the fused pass's two tile shapes: variant 1
// (1024-event tiles, two CTAs per SM; its cost grows with the partition like
// Eq. 6's CPU cost) and variant 2 (2048-event tiles; fewer partial groups per
// event, its relative cost falls with the partition like Eq. 7's GPU cost).
// Part = batch bytes / partitions (the SMs).  The inflection point where the
// two cost the same is refitted after every batch by Eq. 9 on (throughput,
// latency, observed InfPT) samples, where the observed InfPT is the crossover
// of the two variants' measured costs (power laws ms = c rows^b fitted by
// least squares on logs over their latest samples).
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

struct lms_variant_analytic {
  int partitions = 148;
  double bpr = 16.0;            // bytes per row
  double infpt = 150.0 * 1024;  // inflection point, bytes per partition
  lms_regressor* reg = nullptr;
  int window = 16;              // samples per variant in its cost fit
  int explore = 2;              // each variant is tried this many times first
  std::deque<double> lr[2], lm[2];  // ln rows, ln ms of variants 1 and 2
  double max_thput = 0.0, sum_lat = 0.0;
  long long n_obs = 0;
  long long picks[2] = {0, 0};
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

lms_status lms_admission_truncate(lms_admission* a, int32_t n_keep, double last_bytes) {
  if (!a || a->admitted.empty() || n_keep < 1 || n_keep > (int32_t)a->admitted.size())
    return LMS_EINVAL;
  a->admitted.resize((size_t)n_keep);
  if (last_bytes > 0) a->admitted.back().bytes = last_bytes;
  return LMS_OK;
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

namespace {

// ln ms = a + b ln rows over the samples of one variant (least squares);
// false without two distinct sizes.
bool power_fit(const std::deque<double>& x, const std::deque<double>& y, double* a, double* b) {
  const size_t n = x.size();
  if (n < 2) return false;
  double mx = 0, my = 0;
  for (size_t k = 0; k < n; ++k) {
    mx += x[k];
    my += y[k];
  }
  mx /= (double)n;
  my /= (double)n;
  double sxx = 0, sxy = 0;
  for (size_t k = 0; k < n; ++k) {
    sxx += (x[k] - mx) * (x[k] - mx);
    sxy += (x[k] - mx) * (y[k] - my);
  }
  if (!(sxx > 1e-12)) return false;
  *b = sxy / sxx;
  *a = my - *b * mx;
  return true;
}

}  // namespace

lms_variant_analytic* lms_variant_analytic_create(int32_t partitions, double bytes_per_row,
                                                  double infpt0_bytes, int32_t history_len,
                                                  int32_t explore) {
  if (partitions < 1 || !(bytes_per_row > 0) || !(infpt0_bytes > 0) || history_len < 0 ||
      explore < 0)
    return nullptr;
  lms_variant_analytic* v = new lms_variant_analytic();
  v->partitions = partitions;
  v->bpr = bytes_per_row;
  v->infpt = infpt0_bytes;
  v->explore = explore;
  v->reg = lms_regressor_create(history_len);
  return v;
}

void lms_variant_analytic_destroy(lms_variant_analytic* v) {
  if (!v) return;
  lms_regressor_destroy(v->reg);
  delete v;
}

int32_t lms_variant_analytic_choose(void* ctx, int64_t rows, int32_t n_queries) {
  lms_variant_analytic* v = static_cast<lms_variant_analytic*>(ctx);
  (void)n_queries;
  int32_t pick;
  if ((int)v->lr[0].size() < v->explore || (int)v->lr[1].size() < v->explore) {
    pick = v->lr[0].size() <= v->lr[1].size() ? 1 : 2;  // explore: the less sampled variant
  } else {
    // Alg. 2 over the one-operation chain (Aggregation): variant 1 stands
    // where the paper puts the CPU, variant 2 where it puts the GPU
    const int32_t op = LMS_QOP_AGGREGATION;
    int32_t dev = 0;
    const double bytes = (double)std::max<int64_t>(rows, 1) * v->bpr;
    if (lms_map_device(&op, 1, bytes, v->partitions, v->infpt, 0.1, &dev, nullptr, nullptr) !=
        LMS_OK)
      dev = 0;
    pick = dev == 1 ? 1 : 2;
  }
  ++v->picks[pick - 1];
  return pick;
}

void lms_variant_analytic_observe(void* ctx, int64_t rows, int32_t variant, double ms) {
  lms_variant_analytic* v = static_cast<lms_variant_analytic*>(ctx);
  if (!v || rows < 1 || !(ms > 0) || (variant != 1 && variant != 2)) return;
  const int i = variant - 1;
  v->lr[i].push_back(std::log((double)rows));
  v->lm[i].push_back(std::log(ms));
  if ((int)v->lr[i].size() > v->window) {
    v->lr[i].pop_front();
    v->lm[i].pop_front();
  }
  const double thput = (double)rows / ms, lat = ms;
  v->max_thput = std::max(v->max_thput, thput);
  v->sum_lat += lat;
  ++v->n_obs;
  double a1, b1, a2, b2;
  if (!power_fit(v->lr[0], v->lm[0], &a1, &b1) || !power_fit(v->lr[1], v->lm[1], &a2, &b2)) return;
  // observed InfPT: where the two fits cross, kept within the sizes seen (a
  // factor 2 beyond them when one variant is the cheaper one throughout)
  double lo = 1e300, hi = -1e300;
  for (int k = 0; k < 2; ++k)
    for (double x : v->lr[k]) {
      lo = std::min(lo, x);
      hi = std::max(hi, x);
    }
  lo -= std::log(2.0);
  hi += std::log(2.0);
  double x;
  if (b1 != b2) x = (a1 - a2) / (b2 - b1);
  else x = a1 < a2 ? hi : lo;
  if (x < lo || x > hi) x = (a1 + b1 * hi < a2 + b2 * hi) ? hi : lo;
  const double obs = std::exp(x) * v->bpr / (double)v->partitions;
  lms_regressor_add(v->reg, thput, lat, obs);
  double beta[3], inf = 0.0;
  lms_regressor_fit(v->reg, v->max_thput, v->sum_lat / (double)v->n_obs, beta, &inf);
  if (inf > 0) v->infpt = inf;
}

double lms_variant_analytic_predict(const lms_variant_analytic* v, int64_t rows, int32_t variant) {
  if (!v || rows < 1 || (variant != 1 && variant != 2)) return -1.0;
  double a, b;
  if (!power_fit(v->lr[variant - 1], v->lm[variant - 1], &a, &b)) return -1.0;
  return std::exp(a + b * std::log((double)rows));
}

void lms_variant_analytic_state(const lms_variant_analytic* v, double* infpt_bytes,
                                int64_t* picks) {
  if (!v) return;
  if (infpt_bytes) *infpt_bytes = v->infpt;
  if (picks) {
    picks[0] = v->picks[0];
    picks[1] = v->picks[1];
  }
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

lms_status lms_regressor_fit(lms_regressor* r, double target_thput, double target_lat,
                             double* beta, double* infpt) {
  if (!r || !beta || !infpt) return LMS_EINVAL;
  const size_t n = r->thp.size();
  if (n == 0) {
    beta[0] = 150.0 * 1024.0;
    beta[1] = beta[2] = 0.0;
  } else {
    // least squares with an intercept, on centred inputs
    double mt = 0, ml = 0, my = 0;
    for (size_t k = 0; k < n; ++k) {
      mt += r->thp[k];
      ml += r->lat[k];
      my += r->inf[k];
    }
    mt /= (double)n;
    ml /= (double)n;
    my /= (double)n;
    double stt = 0, sll = 0, stl = 0, sty = 0, sly = 0;
    for (size_t k = 0; k < n; ++k) {
      const double tc = r->thp[k] - mt, lc = r->lat[k] - ml, yc = r->inf[k] - my;
      stt += tc * tc;
      sll += lc * lc;
      stl += tc * lc;
      sty += tc * yc;
      sly += lc * yc;
    }
    const bool degenerate =
        n < 3 || stt == 0.0 || sll == 0.0 || 1.0 - stl * stl / (stt * sll) < 1e-12;
    if (degenerate) {
      beta[0] = my;
      beta[1] = beta[2] = 0.0;
    } else {
      const double det = stt * sll - stl * stl;
      beta[1] = (sty * sll - sly * stl) / det;
      beta[2] = (sly * stt - sty * stl) / det;
      beta[0] = my - beta[1] * mt - beta[2] * ml;
    }
  }
  *infpt = beta[0] + beta[1] * target_thput + beta[2] * target_lat;
  return n < 3 ? LMS_EAGAIN : LMS_OK;
}

}  // extern "C"
