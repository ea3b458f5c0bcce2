// Features of the learned cost model and the Alg. 1 predictor it backs.
//
// The predictor keeps the paper's analytic estimate (Eq. 5: bytes over the
// average throughput of Eq. 3, from the batches it has observed) both as a
// fallback and as the judge of the network: after every batch it compares the
// two predictions of that batch's processing time with the measured one
// (exponential moving average of |ln(predicted / measured)|) and answers with
// the network only once it has been fitted and while it is the more accurate.
// Observed batches also become training samples (five per batch, one per
// operator) in a ring of the latest LMS_MLP_MAX_BATCH; with online refitting
// on, every refit_every batches the network takes refit_steps Adam steps on
// the ring, and the wall time of that is reported to the serving loop as
// blocking time.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "../../include/lmstream.h"

struct lms_learned {
  lms_mlp* m = nullptr;
  lms_serve_gpu* g = nullptr;
  double key_card = 1, selectivity = 1, panes = 1, nq = 1, slide_ms = 1, poll_ms = 10, bpe = 16;
  std::vector<float> x, t;  // ring of samples
  int count = 0, head = 0;
  long long batches = 0;
  double sum_bytes = 0.0, sum_proc = 0.0;  // Eq. 3
  double err_net = 0.0, err_eq5 = 0.0;     // moving averages of |ln(pred / measured)|
  long long judged = 0;
  bool trained = false;
  int refit_every = 0, refit_steps = 0;
  float lr = 1e-3f;
  long long uses_net = 0, uses_eq5 = 0;
  bool host_input = true;  // the batches' columns come from host memory (H2D is an operator)
};

// Learned chooser of the fused pass's variant: the network predicts the pass's
// time for each variant (operator code LMS_OP_K1_VARIANT(v)); the analytic
// chooser (Alg. 2 around the Eq. 9 inflection point) is the fallback and the
// judge, exactly as Eq. 5 is for the batch-time predictor.
struct lms_variant_learned {
  lms_mlp* m = nullptr;
  lms_variant_analytic* an = nullptr;
  double key_card = 1, selectivity = 1, panes = 1, nq = 1;
  std::vector<float> x, t;
  int count = 0, head = 0;
  bool trained = false;
  int refit_every = 0, refit_steps = 0;
  float lr = 1e-3f;
  long long obs = 0, choices = 0;
  double err_net = 0.0, err_an = 0.0;
  long long judged = 0, uses_net = 0, uses_an = 0;
  long long picks[2] = {0, 0};
};

namespace {

// Sum over the operators (no H2D when the input is already on the device) of
// the network's exp(output) us, in ms, for `nb` batches of `rows` rows plus
// one of `rest` rows (rest = 0: none).
double net_predict_ms(lms_learned* l, double rows, double carried, double span_panes,
                      double nb = 1.0, double rest = 0.0) {
  float x[2 * LMS_N_OPS * LMS_MLP_INPUTS], y[2 * LMS_N_OPS];
  const int op0 = l->host_input ? 0 : 1;
  const int nops = LMS_N_OPS - op0;
  int m = 0;
  for (int part = 0; part < (rest > 0 ? 2 : 1); ++part)
    for (int op = op0; op < LMS_N_OPS; ++op)
      lms_cost_features(part ? rest : rows, carried, l->key_card, l->selectivity, l->panes, l->nq,
                        span_panes, op, x + (m++) * LMS_MLP_INPUTS);
  if (lms_mlp_forward(l->m, x, m, y) != LMS_OK) return -1.0;
  double us = 0.0;
  for (int i = 0; i < m; ++i) us += (i < nops ? nb : 1.0) * std::exp((double)y[i]);
  return us * 1e-3;
}

template <class L>
void push_sample(L* l, const float* x, float t) {
  const int cap = LMS_MLP_MAX_BATCH;
  std::copy(x, x + LMS_MLP_INPUTS, l->x.begin() + (size_t)l->head * LMS_MLP_INPUTS);
  l->t[l->head] = t;
  l->head = (l->head + 1) % cap;
  l->count = std::min(l->count + 1, cap);
}

// The network's fused-pass time of `variant` for `rows` rows, ms (< 0 on error).
double net_variant_ms(lms_variant_learned* v, double rows, int variant) {
  float x[LMS_MLP_INPUTS], y = 0.f;
  lms_cost_features(rows, 0.0, v->key_card, v->selectivity, v->panes, v->nq, 0.0,
                    LMS_OP_K1_VARIANT(variant), x);
  if (lms_mlp_forward(v->m, x, 1, &y) != LMS_OK) return -1.0;
  return std::exp((double)y) * 1e-3;
}

float log_us(double ms) { return (float)std::log(std::max(1.0, ms * 1e3)); }

}  // namespace

extern "C" {

void lms_cost_features(double rows, double carried_groups, double key_card, double selectivity,
                       double panes_per_window, double n_queries, double span_panes, int32_t op,
                       float* out) {
  out[0] = (float)(std::log2(1.0 + std::max(0.0, rows)) / 32.0);
  out[1] = (float)(std::log2(1.0 + std::max(0.0, carried_groups)) / 32.0);
  out[2] = (float)(std::log2(std::max(1.0, key_card)) / 32.0);
  out[3] = (float)selectivity;
  out[4] = (float)(std::log2(std::max(1.0, panes_per_window)) / 12.0);
  out[5] = (float)(n_queries / 8.0);
  out[6] = (float)(std::log2(1.0 + std::max(0.0, span_panes)) / 16.0);
  out[7] = (float)op / 4.0f;
}

lms_learned* lms_learned_create(lms_mlp* m, lms_serve_gpu* g, double key_card, double selectivity,
                                double panes_per_window, double n_queries, double slide_ms,
                                double poll_ms, double bytes_per_event) {
  if (!m || !(slide_ms > 0) || !(poll_ms > 0) || !(bytes_per_event > 0)) return nullptr;
  lms_learned* l = new lms_learned();
  l->m = m;
  l->g = g;
  l->key_card = key_card;
  l->selectivity = selectivity;
  l->panes = panes_per_window;
  l->nq = n_queries;
  l->slide_ms = slide_ms;
  l->poll_ms = poll_ms;
  l->bpe = bytes_per_event;
  l->x.assign((size_t)LMS_MLP_MAX_BATCH * LMS_MLP_INPUTS, 0.f);
  l->t.assign(LMS_MLP_MAX_BATCH, 0.f);
  return l;
}

void lms_learned_destroy(lms_learned* l) { delete l; }

void lms_learned_set_online(lms_learned* l, int32_t refit_every, int32_t refit_steps, float lr) {
  if (!l) return;
  l->refit_every = std::max(0, refit_every);
  l->refit_steps = std::max(0, refit_steps);
  l->lr = lr > 0 ? lr : 1e-3f;
}

void lms_learned_set_backend(lms_learned* l, lms_serve_gpu* g) {
  if (!l) return;
  l->g = g;
  if (!g) return;  // unbinding keeps the last run's judge statistics
  // a new serving run: Eq. 5's history and the judge's errors start afresh
  l->host_input = lms_serve_gpu_device_input(g) == 0;
  l->sum_bytes = l->sum_proc = 0.0;
  l->err_net = l->err_eq5 = 0.0;
  l->judged = 0;
  l->uses_net = l->uses_eq5 = 0;
}

int32_t lms_learned_samples(const lms_learned* l) { return l ? l->count : 0; }

lms_status lms_learned_fit(lms_learned* l, int32_t steps, float lr, float* loss) {
  if (!l || steps < 0) return LMS_EINVAL;
  if (l->count == 0) return LMS_EAGAIN;
  const lms_status r =
      lms_mlp_train(l->m, l->x.data(), l->t.data(), l->count, steps, lr, nullptr, loss);
  if (r == LMS_OK && steps > 0) l->trained = true;
  return r;
}

void lms_learned_stats(const lms_learned* l, double* err_net, double* err_eq5, int64_t* uses_net,
                       int64_t* uses_eq5) {
  if (!l) return;
  if (err_net) *err_net = l->err_net;
  if (err_eq5) *err_eq5 = l->err_eq5;
  if (uses_net) *uses_net = l->uses_net;
  if (uses_eq5) *uses_eq5 = l->uses_eq5;
}

double lms_learned_observe(void* ctx, const lms_serve_batch* rec) {
  lms_learned* l = static_cast<lms_learned*>(ctx);
  if (!l || !rec || rec->n_events <= 0) return 0.0;
  const auto t0 = std::chrono::steady_clock::now();
  const double rows = (double)rec->n_events;
  const double carried = (double)rec->state_groups_before;
  const double span = (double)rec->n_chunks * l->poll_ms / l->slide_ms;
  const double proc = rec->proc_ms;
  // judge: both predictors on this batch against the measured time
  if (proc > 0) {
    const double bytes = rows * l->bpe;
    if (l->trained) {
      const double pn = net_predict_ms(l, rows, carried, span);
      const double pe = l->sum_proc > 0 ? bytes / (l->sum_bytes / l->sum_proc) : -1.0;
      if (pn > 0 && pe > 0) {
        const double a = l->judged < 10 ? 1.0 / (double)(l->judged + 1) : 0.1;
        l->err_net += a * (std::fabs(std::log(pn / proc)) - l->err_net);
        l->err_eq5 += a * (std::fabs(std::log(pe / proc)) - l->err_eq5);
        ++l->judged;
      }
    }
    l->sum_bytes += bytes;
    l->sum_proc += proc;
  }
  // training samples, one per operator
  const double op_ms[LMS_N_OPS] = {
      rec->h2d_ms, rec->k1_ms, rec->sort_ms, rec->emit_ms,
      proc - (rec->h2d_ms + rec->k1_ms + rec->sort_ms + rec->emit_ms)};
  float x[LMS_MLP_INPUTS];
  for (int op = l->host_input ? 0 : 1; op < LMS_N_OPS; ++op) {
    lms_cost_features(rows, carried, l->key_card, l->selectivity, l->panes, l->nq, span, op, x);
    push_sample(l, x, log_us(op_ms[op]));
  }
  ++l->batches;
  if (l->refit_every > 0 && l->refit_steps > 0 && l->batches % l->refit_every == 0)
    lms_learned_fit(l, l->refit_steps, l->lr, nullptr);
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

double lms_learned_predict(void* ctx, double batch_bytes, int32_t n_datasets) {
  lms_learned* l = static_cast<lms_learned*>(ctx);
  const double eq5 = l->sum_proc > 0 ? batch_bytes / (l->sum_bytes / l->sum_proc) : 0.0;
  if (!l->trained || (l->judged >= 5 && l->err_net > l->err_eq5)) {
    ++l->uses_eq5;
    return eq5;  // fallback: the analytic estimate
  }
  double carried = 0.0, cap = -1.0;
  if (l->g) {
    lms_stream* s = lms_serve_gpu_stream(l->g);
    lms_stats st{};
    if (lms_stream_stats(s, &st) == LMS_OK) carried = (double)st.state_groups;
    int64_t adm = -1;
    if (lms_stream_admissible_rows(s, l->host_input ? 1 : 0, &adm) == LMS_OK && adm > 0)
      cap = (double)adm;
  }
  // a candidate larger than the memory admits runs as several capped batches
  const double rows = batch_bytes / l->bpe;
  const double span = (double)n_datasets * l->poll_ms / l->slide_ms;
  double p;
  if (cap > 0 && rows > cap) {
    const double nb = std::floor(rows / cap);
    p = net_predict_ms(l, cap, carried, span * cap / rows, nb, rows - nb * cap);
  } else {
    p = net_predict_ms(l, rows, carried, span);
  }
  if (p < 0) {
    ++l->uses_eq5;
    return eq5;
  }
  ++l->uses_net;
  return p;
}

lms_variant_learned* lms_variant_learned_create(lms_mlp* m, lms_variant_analytic* judge,
                                                double key_card, double selectivity,
                                                double panes_per_window, double n_queries) {
  if (!m || !judge) return nullptr;
  lms_variant_learned* v = new lms_variant_learned();
  v->m = m;
  v->an = judge;
  v->key_card = key_card;
  v->selectivity = selectivity;
  v->panes = panes_per_window;
  v->nq = n_queries;
  v->x.assign((size_t)LMS_MLP_MAX_BATCH * LMS_MLP_INPUTS, 0.f);
  v->t.assign(LMS_MLP_MAX_BATCH, 0.f);
  return v;
}

void lms_variant_learned_destroy(lms_variant_learned* v) { delete v; }

void lms_variant_learned_set_online(lms_variant_learned* v, int32_t refit_every,
                                    int32_t refit_steps, float lr) {
  if (!v) return;
  v->refit_every = std::max(0, refit_every);
  v->refit_steps = std::max(0, refit_steps);
  v->lr = lr > 0 ? lr : 1e-3f;
}

lms_status lms_variant_learned_fit(lms_variant_learned* v, int32_t steps, float lr, float* loss) {
  if (!v || steps < 0) return LMS_EINVAL;
  if (v->count == 0) return LMS_EAGAIN;
  const lms_status r =
      lms_mlp_train(v->m, v->x.data(), v->t.data(), v->count, steps, lr, nullptr, loss);
  if (r == LMS_OK && steps > 0) v->trained = true;
  return r;
}

int32_t lms_variant_learned_choose(void* ctx, int64_t rows, int32_t n_queries) {
  lms_variant_learned* v = static_cast<lms_variant_learned*>(ctx);
  ++v->choices;
  // the analytic recommendation (it also explores both variants first)
  const int32_t an_pick = lms_variant_analytic_choose(v->an, rows, n_queries);
  int32_t pick = an_pick;
  const bool net_ok = v->trained && !(v->judged >= 5 && v->err_net > v->err_an);
  if (net_ok) {
    const double p1 = net_variant_ms(v, (double)rows, 1), p2 = net_variant_ms(v, (double)rows, 2);
    if (p1 > 0 && p2 > 0) {
      pick = p1 <= p2 ? 1 : 2;
      if (v->choices % 16 == 0) pick = 3 - pick;  // keep measuring the other variant
      ++v->uses_net;
    } else {
      ++v->uses_an;
    }
  } else {
    ++v->uses_an;
  }
  ++v->picks[pick - 1];
  return pick;
}

void lms_variant_learned_observe(void* ctx, int64_t rows, int32_t variant, double ms) {
  lms_variant_learned* v = static_cast<lms_variant_learned*>(ctx);
  if (!v || rows < 1 || !(ms > 0) || (variant != 1 && variant != 2)) return;
  // judge both models on this pass before either learns from it
  if (v->trained) {
    const double pn = net_variant_ms(v, (double)rows, variant);
    const double pa = lms_variant_analytic_predict(v->an, rows, variant);
    if (pn > 0 && pa > 0) {
      const double a = v->judged < 10 ? 1.0 / (double)(v->judged + 1) : 0.1;
      v->err_net += a * (std::fabs(std::log(pn / ms)) - v->err_net);
      v->err_an += a * (std::fabs(std::log(pa / ms)) - v->err_an);
      ++v->judged;
    }
  }
  lms_variant_analytic_observe(v->an, rows, variant, ms);
  float x[LMS_MLP_INPUTS];
  lms_cost_features((double)rows, 0.0, v->key_card, v->selectivity, v->panes, v->nq, 0.0,
                    LMS_OP_K1_VARIANT(variant), x);
  push_sample(v, x, log_us(ms));
  ++v->obs;
  if (v->refit_every > 0 && v->refit_steps > 0 && v->obs % v->refit_every == 0)
    lms_variant_learned_fit(v, v->refit_steps, v->lr, nullptr);
}

void lms_variant_learned_stats(const lms_variant_learned* v, double* err_net, double* err_an,
                               int64_t* uses_net, int64_t* uses_an, int64_t* picks) {
  if (!v) return;
  if (err_net) *err_net = v->err_net;
  if (err_an) *err_an = v->err_an;
  if (uses_net) *uses_net = v->uses_net;
  if (uses_an) *uses_an = v->uses_an;
  if (picks) {
    picks[0] = v->picks[0];
    picks[1] = v->picks[1];
  }
}

}  // extern "C"
