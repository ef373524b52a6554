// grt_api.cu -- the C ABI of libgrt (declared in include/grt.h).
//
// Host work only: argument validation, the branching-law tables, the
// (point, tree-tile) work layout, device buffers, and the launches of the
// walk and finalize kernels.  Every step of the solve itself runs on the GPU.
#include "grt.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "grt_device.cuh"
#include "grt_host.h"
#include "grt_launch.h"

namespace {

thread_local std::string g_create_error;



// Threshold of a cumulative probability on the 32-bit word scale:
// round-to-nearest of 2^32 * cum, clamped to [0, 2^32].
uint64_t word_threshold(double cum) {
  const double v = cum * 4294967296.0;
  if (v <= 0.0) return 0;
  if (v >= 4294967296.0) return 4294967296ull;
  return (uint64_t)llround(v);
}

bool is_finite(double v) { return std::isfinite(v); }

}  // namespace

struct grt_plan {
  grt_ctx *ctx = nullptr;
  int64_t n = 0;
  int K = 0, L = 0, M = 0;
  uint32_t total_items = 0;
  uint64_t total_trees = 0;
  std::vector<uint64_t> host_ntrees;
  uint32_t total_chunks = 0;
  grt::DevBuf prefix, tree_prefix, ntrees, rec_w, rec_o, chunk_prefix, part;
  grt::DevBuf work;  // queue head (8 B), 3 u64 counters, then n u32 chunk tickets
  size_t work_bytes = 64;
  cudaStream_t last_stream = nullptr;
  bool executed = false;  // an execution (or graph replay) has been enqueued: the chunk sums exist
  int launches = 0;
  bool timing = false, timed_last = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  grt::WalkConfig cfg{};             // launch shape of the walk (autotuned or set)
  uint32_t tile_small = 0;           // queue chunk of points small_from .. n-1 (0: none)
  int64_t small_from = 0;
  // walk launches: points [group_pt[g], group_pt[g+1]), whose records span fewer than 2^32 slots
  // (one group unless the plan holds that many records)
  std::vector<int64_t> group_pt;
  std::vector<uint32_t> group_item;        // first queue item of each group (and the end)
  std::vector<unsigned long long> group_rec;  // first record slot of each group
  cudaGraph_t graph = nullptr;       // a captured execution (grt_plan_graph_capture)
  cudaGraphExec_t graph_exec = nullptr;
  void release() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    graph_exec = nullptr;
    graph = nullptr;
    for (auto &e : ev)
      if (e) {
        cudaEventDestroy(e);
        e = nullptr;
      }
    prefix.release();
    tree_prefix.release();
    ntrees.release();
    rec_w.release();
    rec_o.release();
    chunk_prefix.release();
    part.release();
    work.release();
  }
};

namespace {



// Validate the problem and build the walk's tables (branching law of
// Sec. 2.1 Eq. probexp2 / Sec. 2.2 Eq. probexpB1 on 32-bit thresholds).
int build_tables(const grt_problem &pb, grt::WalkParams &w, std::string &why) {
  if (pb.dim < 1 || pb.dim > GRT_MAX_DIM) return why = "dim must be 1, 2 or 3", GRT_EINVAL;
  if (!is_finite(pb.D) || pb.D < 0.0) return why = "D must be finite and >= 0", GRT_EINVAL;
  if (pb.f_deg < 0 || pb.f_deg > GRT_MAX_DEG) return why = "f_deg must be in [0, 15]", GRT_EINVAL;
  for (int k = 0; k <= pb.f_deg; ++k)
    if (!is_finite(pb.f_coef[k])) return why = "f_coef must be finite", GRT_EINVAL;
  if (pb.u0_kind < GRT_U0_CONST || pb.u0_kind > GRT_U0_QUADRATIC) return why = "unknown u0_kind", GRT_EINVAL;
  if (pb.sde_kind != GRT_SDE_HEAT && pb.sde_kind != GRT_SDE_AFFINE) return why = "unknown sde_kind", GRT_EINVAL;
  if (pb.sde_kind == GRT_SDE_AFFINE) {
    if (pb.sde_steps < 1 || pb.sde_steps > 4096) return why = "sde_steps must be in [1, 4096]", GRT_EINVAL;
    for (int i = 0; i < 12; ++i)
      if (!is_finite(pb.sde_param[i])) return why = "sde_param must be finite", GRT_EINVAL;
  }
  for (int i = 0; i < 8; ++i)
    if (!is_finite(pb.u0_param[i])) return why = "u0_param must be finite", GRT_EINVAL;
  if (pb.u0_kind == GRT_U0_GAUSS && pb.u0_param[2] == 0.0) return why = "GAUSS width p2 must be nonzero", GRT_EINVAL;
  if (pb.u0_kind == GRT_U0_LOGISTIC && pb.u0_param[3] == 0.0)
    return why = "LOGISTIC width p3 must be nonzero", GRT_EINVAL;
  if (pb.strategy != GRT_STRATEGY_A && pb.strategy != GRT_STRATEGY_B) return why = "unknown strategy", GRT_EINVAL;
  if (pb.arity_law != GRT_ARITY_UNIFORM && pb.arity_law != GRT_ARITY_ABS_COEF)
    return why = "unknown arity_law", GRT_EINVAL;
  if (pb.precision != GRT_FP32 && pb.precision != GRT_FP64) return why = "unknown precision", GRT_EINVAL;
  const bool A = pb.strategy == GRT_STRATEGY_A;
  if (A && !(is_finite(pb.lambda) && pb.lambda > 0.0)) return why = "Strategy A needs lambda > 0", GRT_EINVAL;
  if (A && !is_finite(pb.c_pot)) return why = "c_pot must be finite", GRT_EINVAL;
  if (!A && !(pb.q > 0.0 && pb.q < 1.0)) return why = "Strategy B needs 0 < q < 1", GRT_EINVAL;
  if (pb.coef_kind < GRT_COEF_CONST || pb.coef_kind > GRT_COEF_GAUSS) return why = "unknown coef_kind", GRT_EINVAL;
  const bool varcoef = pb.coef_kind != GRT_COEF_CONST;
  if (varcoef) {
    for (int i = 0; i < 8; ++i)
      if (!is_finite(pb.coef_param[i])) return why = "coef_param must be finite", GRT_EINVAL;
    if (pb.coef_kind == GRT_COEF_GAUSS_OVER_T && !(pb.coef_param[6] > 0.0))
      return why = "GAUSS_OVER_T needs t0 = coef_param[6] > 0", GRT_EINVAL;
    if (A && pb.c_pot != 0.0 && ((pb.coef_mask >> 1) & 1u))
      return why = "a variable linear coefficient cannot be combined with c_pot != 0 (Strategy A)", GRT_EINVAL;
  }

  // Terms: the nonzero coefficients of F = f + c u (A) or f (B), by ascending power.
  const int deg = (A && pb.f_deg < 1) ? 1 : pb.f_deg;
  double F[GRT_MAX_DEG + 1];
  for (int k = 0; k <= deg; ++k) F[k] = (k <= pb.f_deg ? pb.f_coef[k] : 0.0) + ((A && k == 1) ? pb.c_pot : 0.0);
  int nt = 0;
  double coef[grt::kMaxTerms];
  for (int k = 0; k <= deg; ++k) {
    if (F[k] != 0.0) {
      w.arity[nt] = k;
      coef[nt] = F[k];
      ++nt;
    }
  }
  w.nterms = nt;
  // variable coefficients: the categories (term indices) whose power is in the mask
  w.coef_kind = pb.coef_kind;
  w.coef_cat_mask = 0u;
  for (int i = 0; i < 3; ++i) {
    w.cwd[i] = varcoef ? -pb.coef_param[i] : 0.0;
    w.cmd[i] = varcoef ? pb.coef_param[3 + i] : 0.0;
    w.cwf[i] = (float)(w.cwd[i] * 1.4426950408889634);
  }
  w.ct0d = varcoef ? pb.coef_param[6] : 0.0;
  w.sde_kind = pb.sde_kind;
  w.sde_steps = pb.sde_kind == GRT_SDE_AFFINE ? pb.sde_steps : 0;
  for (int i = 0; i < 12; ++i) {
    w.sded[i] = pb.sde_kind == GRT_SDE_AFFINE ? pb.sde_param[i] : 0.0;
    w.sdef[i] = (float)w.sded[i];
  }
  w.ct0f = (float)w.ct0d;
  if (varcoef)
    for (int i = 0; i < nt; ++i)
      if ((pb.coef_mask >> w.arity[i]) & 1u) w.coef_cat_mask |= 1u << i;
  for (int i = nt; i < grt::kMaxTerms; ++i) {
    w.arity[i] = 0;
    w.term_factor[i] = 0.0;
  }
  double prob[grt::kMaxTerms];
  double sabs = 0.0;
  for (int i = 0; i < nt; ++i) sabs += std::fabs(coef[i]);
  for (int i = 0; i < nt; ++i)
    prob[i] = pb.arity_law == GRT_ARITY_ABS_COEF ? std::fabs(coef[i]) / sabs : 1.0 / (double)nt;

  uint64_t T[grt::kMaxTerms + 1];
  int ncat = 0;
  if (!A) {
    // joint draw over {leaf, term 1..nt}: P(leaf) = q, P(term i) = (1 - q) p_i
    if (nt == 0) {
      T[0] = 4294967296ull;
      ncat = 1;
      w.leaf_factor = 1.0;
    } else {
      T[0] = word_threshold(pb.q);
      double cp = 0.0;
      for (int i = 0; i < nt; ++i) {
        cp += prob[i];
        T[i + 1] = word_threshold(pb.q + (1.0 - pb.q) * cp);
      }
      T[nt] = 4294967296ull;
      ncat = nt + 1;
      if (T[0] == 0) return why = "q too small for a 32-bit leaf threshold", GRT_EINVAL;
      w.leaf_factor = 4294967296.0 / (double)T[0];
      for (int i = 0; i < nt; ++i) {
        const double P = (double)(T[i + 1] - T[i]) / 4294967296.0;
        w.term_factor[i] = P > 0.0 ? coef[i] / P : 0.0;
      }
    }
  } else {
    w.leaf_factor = 1.0;
    if (nt > 0) {
      double cp = 0.0;
      for (int i = 0; i < nt; ++i) {
        cp += prob[i];
        T[i] = word_threshold(cp);
      }
      T[nt - 1] = 4294967296ull;
      ncat = nt;
      for (int i = 0; i < nt; ++i) {
        const double P = (double)(T[i] - (i == 0 ? 0ull : T[i - 1])) / 4294967296.0;
        w.term_factor[i] = P > 0.0 ? coef[i] / (pb.lambda * P) : 0.0;
      }
    }
  }
  w.leaf_factorf = (float)w.leaf_factor;
  // finite thresholds: all before the first that reaches 2^32
  int nfin = 0;
  while (nfin < ncat - 1 && T[nfin] < 4294967296ull) ++nfin;
  w.ncat_thr = nfin;
  for (int j = 0; j <= grt::kMaxTerms; ++j) w.thr[j] = j < nfin ? (uint32_t)T[j] : 0xFFFFFFFFu;

  // problem scalars
  w.u0_kind = pb.u0_kind;
  w.two_D = 2.0 * pb.D;
  w.inv_lambda = A ? 1.0 / pb.lambda : 1.0;
  w.lam_minus_c = A ? pb.lambda - pb.c_pot : 0.0;
  w.two_Df = (float)w.two_D;
  w.inv_lambdaf = (float)w.inv_lambda;
  w.lam_minus_cf = (float)w.lam_minus_c;
  const double *a = pb.u0_param;
  double c[8] = {a[0], a[1], 0, 0, 0, 0, 0, 0};
  switch (pb.u0_kind) {
  case GRT_U0_GAUSS:
    c[2] = -1.0 / (2.0 * a[2] * a[2]);
    c[3] = a[3];
    c[4] = a[4];
    c[5] = a[5];
    break;
  case GRT_U0_COS_PROD:
  case GRT_U0_TANH_PROD:
    c[2] = a[2];
    c[3] = a[3];
    c[4] = a[4];
    break;
  case GRT_U0_LOGISTIC:
    c[2] = a[2];
    c[3] = -1.0 / a[3];
    break;
  case GRT_U0_GAUSS_AXES:
    for (int i = 0; i < 3; ++i) {
      c[2 + i] = -a[2 + i];
      c[5 + i] = a[5 + i];
    }
    break;
  case GRT_U0_QUADRATIC:
    for (int i = 1; i < 7; ++i) c[i] = a[i];
    break;
  default:
    break;
  }
  // FP32 copy: exponent scales carry log2(e) (the FP32 walk evaluates e^v as 2^(v log2 e))
  const double log2e = 1.4426950408889634;
  for (int i = 0; i < 8; ++i) {
    w.u0d[i] = c[i];
    w.u0f[i] = (float)c[i];
  }
  if (pb.u0_kind == GRT_U0_GAUSS) w.u0f[2] = (float)(c[2] * log2e);
  if (pb.u0_kind == GRT_U0_LOGISTIC) w.u0f[3] = (float)(c[3] * log2e);
  if (pb.u0_kind == GRT_U0_GAUSS_AXES)
    for (int i = 2; i < 5; ++i) w.u0f[i] = (float)(c[i] * log2e);
  w.lam_minus_cf = (float)(w.lam_minus_c * log2e);
  return GRT_OK;
}

void set_round_keys(grt::WalkParams &w, uint64_t seed) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    w.rk0[r] = k0;
    w.rk1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

size_t acc_size(const grt_ctx *c) { return c->pb.precision == GRT_FP64 ? sizeof(double) : sizeof(float); }

// Lay out the work items of a plan and size its buffers (grow only).
int plan_configure(grt_plan *p, int64_t n, const uint64_t *ntrees, int K, int L, int M) {
  grt_ctx *c = p->ctx;
  if (n < 0 || n > 0x7FFFFFFFll) return c->set_error(GRT_EINVAL, "n must be in [0, 2^31)");
  if (K < 0 || K > GRT_MAX_K) return c->set_error(GRT_EINVAL, "K must be in [0, 16]");
  if (L < 0 || M < 0 || L + M > K) return c->set_error(GRT_EINVAL, "need L, M >= 0 and L + M <= K");
  if (n > 0 && !ntrees) return c->set_error(GRT_EINVAL, "ntrees is NULL");
  const bool same = p->n == n && p->K == K && p->host_ntrees.size() == (size_t)n &&
                    (n == 0 || std::memcmp(p->host_ntrees.data(), ntrees, (size_t)n * sizeof(uint64_t)) == 0);
  if (same && p->prefix.ptr) {
    p->L = L;
    p->M = M;
    return GRT_OK;
  }
  p->n = -1;  // invalid until the new layout is complete
  p->host_ntrees.clear();
  std::vector<uint32_t> prefix((size_t)n + 1), nt32((size_t)n);
  std::vector<unsigned long long> tprefix((size_t)n + 1);
  std::vector<uint32_t> cprefix((size_t)n + 1);
  uint64_t items = 0, trees = 0, chunks = 0, recs = 0;  // recs: record slots, each point's segment 4-aligned
  // the points at the end of the queue, about its last 1/32 of the trees (when that is at most 1/16
  // of them), are cut into 64-tree chunks: a warp that finds the queue empty then waits only for
  // short chunks of the others, at the cost of more chunk fetches on a small share of the trees
  uint64_t all = 0;
  for (int64_t i = 0; i < n; ++i) all += ntrees[i];
  p->tile_small = 0;
  p->small_from = n;
  if (p->cfg.tile > 64 && n > 1) {
    uint64_t tail = 0;
    int64_t i = n;
    while (i > 1 && tail < all / 32) tail += ntrees[--i];
    if (tail <= all / 16) {
      p->tile_small = 64;
      p->small_from = i;
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    if (ntrees[i] > GRT_MAX_TREES_PER_POINT) return c->set_error(GRT_EINVAL, "ntrees[i] above 2^31 - 1");
    const uint64_t tl = (p->tile_small != 0 && i >= p->small_from) ? p->tile_small : p->cfg.tile;
    prefix[(size_t)i] = (uint32_t)items;
    tprefix[(size_t)i] = recs;
    recs += (ntrees[i] + 3) & ~(uint64_t)3;
    cprefix[(size_t)i] = (uint32_t)chunks;
    chunks += ntrees[i] == 0 ? 1 : (ntrees[i] + grt::kBinChunk - 1) / grt::kBinChunk;
    items += (ntrees[i] + tl - 1) / tl;
    trees += ntrees[i];
    nt32[(size_t)i] = (uint32_t)ntrees[i];
    if (items >= 0xFFFFFFFFull) return c->set_error(GRT_EINVAL, "too many work items (total trees too large)");
  }
  prefix[(size_t)n] = (uint32_t)items;
  tprefix[(size_t)n] = recs;
  cprefix[(size_t)n] = (uint32_t)chunks;
  if (chunks > 0x7FFFFFFFull) return c->set_error(GRT_EINVAL, "too many binning chunks (total trees too large)");
  GRT_CUDA(c, cudaSetDevice(c->device));
  GRT_CUDA(c, p->prefix.ensure(prefix.size() * sizeof(uint32_t)));
  GRT_CUDA(c, p->tree_prefix.ensure(tprefix.size() * sizeof(unsigned long long)));
  GRT_CUDA(c, p->ntrees.ensure(nt32.size() * sizeof(uint32_t) + 4));
  GRT_CUDA(c, p->rec_w.ensure((size_t)recs * acc_size(c) + 64));
  GRT_CUDA(c, p->rec_o.ensure((size_t)recs + 64));
  GRT_CUDA(c, p->chunk_prefix.ensure(cprefix.size() * sizeof(uint32_t)));
  GRT_CUDA(c, p->part.ensure((size_t)chunks * 4 * (K + 2) * sizeof(double) + 16));
  p->work_bytes = 64 + (((size_t)n * sizeof(uint32_t) + 63) & ~(size_t)63);
  GRT_CUDA(c, p->work.ensure(p->work_bytes));
  GRT_CUDA(c, cudaMemcpy(p->prefix.ptr, prefix.data(), prefix.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  GRT_CUDA(c, cudaMemcpy(p->tree_prefix.ptr, tprefix.data(), tprefix.size() * sizeof(unsigned long long),
                         cudaMemcpyHostToDevice));
  if (n > 0)
    GRT_CUDA(c, cudaMemcpy(p->ntrees.ptr, nt32.data(), nt32.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  GRT_CUDA(c, cudaMemcpy(p->chunk_prefix.ptr, cprefix.data(), cprefix.size() * sizeof(uint32_t),
                         cudaMemcpyHostToDevice));
  GRT_CUDA(c, cudaMemset(p->work.ptr, 0, p->work_bytes));
  // walk launch groups: consecutive points whose record slots span fewer than `window`
  unsigned long long window = 0xFFFFFFFFull;
  if (const char *ev = std::getenv("GRT_MAX_RECORDS_PER_LAUNCH")) {  // testing aid: smaller windows
    const unsigned long long v = std::strtoull(ev, nullptr, 10);
    if (v >= 4096 && v < window) window = v;
  }
  p->group_pt.assign(1, 0);
  p->group_item.assign(1, 0);
  p->group_rec.assign(1, 0);
  for (int64_t i = 0; i < n; ++i) {
    const unsigned long long seg_end = tprefix[(size_t)i + 1];
    if (seg_end - p->group_rec.back() > window && i > p->group_pt.back()) {
      p->group_pt.push_back(i);
      p->group_item.push_back(prefix[(size_t)i]);
      p->group_rec.push_back(tprefix[(size_t)i]);
    }
    if (seg_end - p->group_rec.back() > 0xFFFFFFFFull)
      return c->set_error(GRT_EINVAL, "one point's records span 2^32 slots");
  }
  p->group_pt.push_back(n);
  p->group_item.push_back((uint32_t)items);
  p->total_chunks = (uint32_t)chunks;
  p->n = n;
  p->K = K;
  p->L = L;
  p->M = M;
  p->total_items = (uint32_t)items;
  p->total_trees = trees;
  p->host_ntrees.assign(ntrees, ntrees + n);
  p->launches = (items > 0 ? (int)(p->group_pt.size() - 1) : 0) + 2;  // walk launch(es), binning, completion
  return GRT_OK;
}

int plan_execute(grt_plan *p, const double *d_x, const double *d_t, uint64_t seed, uint64_t point_base, double *d_u,
                 double *d_coef, double *d_se, int32_t *d_status, cudaStream_t stream) {
  grt_ctx *c = p->ctx;
  if (p->n < 0) return c->set_error(GRT_EINVAL, "plan has no valid layout (its last configuration failed)");
  if (p->n == 0) return GRT_OK;
  if (!d_x || !d_t || !d_u) return c->set_error(GRT_EINVAL, "x, t and u must be non-NULL");
  if (point_base + (uint64_t)p->n - 1 > 0xFFFFFFFFull) return c->set_error(GRT_EINVAL, "point_base + n exceeds 2^32");
  GRT_CUDA(c, cudaSetDevice(c->device));
  grt::WalkParams w = c->base;
  set_round_keys(w, seed);
  w.K = p->K;
  w.point_base = (uint32_t)point_base;
  w.x = d_x;
  w.t = d_t;
  w.ntrees = p->ntrees.as<uint32_t>();
  w.prefix = p->prefix.as<uint32_t>();
  w.tree_prefix = p->tree_prefix.as<unsigned long long>();
  w.n = (int)p->n;
  w.tile = p->cfg.tile;
  w.tile_small = p->tile_small;
  w.small_from = (int)p->small_from;
  w.total_items = p->total_items;
  w.rec_w = p->rec_w.ptr;
  w.rec_o = p->rec_o.as<uint8_t>();
  w.counter = p->work.as<uint32_t>();
  w.stats = reinterpret_cast<unsigned long long *>(p->work.as<unsigned char>() + 8);
  const bool fp64 = c->pb.precision == GRT_FP64;
  if (p->timing) GRT_CUDA(c, cudaEventRecord(p->ev[0], stream));
  GRT_CUDA(c, cudaMemsetAsync(p->work.ptr, 0, p->work_bytes, stream));
  for (size_t g = 0; g + 1 < p->group_pt.size() && p->total_items > 0; ++g) {
    if (p->group_item[g + 1] == p->group_item[g]) continue;  // no trees in this group
    if (g > 0) GRT_CUDA(c, cudaMemsetAsync(p->work.ptr, 0, sizeof(uint32_t), stream));  // queue head
    w.n = (int)p->group_pt[g + 1];  // the point search covers points below the group's end
    w.item_base = p->group_item[g];
    w.total_items = p->group_item[g + 1];
    w.rec_base = p->group_rec[g];
    w.rec_w = static_cast<unsigned char *>(p->rec_w.ptr) + (size_t)p->group_rec[g] * acc_size(c);
    w.rec_o = p->rec_o.as<uint8_t>() + p->group_rec[g];
    GRT_CUDA(c, grt::launch_walk(fp64, c->pb.dim, c->pb.strategy, w, p->cfg, c->num_sms, stream));
  }
  if (p->timing) GRT_CUDA(c, cudaEventRecord(p->ev[1], stream));
  grt::FinalizeParams f{};
  f.rec_w = p->rec_w.ptr;
  f.rec_o = p->rec_o.as<uint8_t>();
  f.tree_prefix = p->tree_prefix.as<unsigned long long>();
  f.ntrees = p->ntrees.as<uint32_t>();
  f.chunk_prefix = p->chunk_prefix.as<uint32_t>();
  f.total_chunks = p->total_chunks;
  f.part = p->part.as<double>();
  f.n = (int)p->n;
  f.K = p->K;
  f.stats = w.stats;
  GRT_CUDA(c, grt::launch_finalize(fp64, f, stream));
  // each point's chunk sums -> a_n, SE_n, Pade
  grt::CompleteParams cp{};
  cp.n = (int)p->n;
  cp.K = p->K;
  cp.L = p->L;
  cp.M = p->M;
  cp.part = p->part.as<double>();
  cp.chunk_prefix = p->chunk_prefix.as<uint32_t>();
  cp.ntrees = p->ntrees.as<uint32_t>();
  cp.u = d_u;
  cp.coef = d_coef;
  cp.se = d_se;
  cp.status = d_status;
  GRT_CUDA(c, grt::launch_complete(cp, stream));
  if (p->timing) GRT_CUDA(c, cudaEventRecord(p->ev[2], stream));
  p->timed_last = p->timing;
  p->last_stream = stream;
  p->executed = true;
  return GRT_OK;
}

}  // namespace

extern "C" {

int grt_create(const grt_problem *pb, int device, grt_ctx **out) {
  if (!out) return GRT_EINVAL;
  *out = nullptr;
  if (!pb) {
    g_create_error = "problem is NULL";
    return GRT_EINVAL;
  }
  grt::WalkParams w{};
  std::string why;
  int rc = build_tables(*pb, w, why);
  if (rc != GRT_OK) {
    g_create_error = why;
    return rc;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return GRT_EDEVICE;
  }
  if (device < 0 || device >= ndev) {
    g_create_error = "device index out of range";
    return GRT_EINVAL;
  }
  grt_ctx *c = new (std::nothrow) grt_ctx();
  if (!c) {
    g_create_error = "out of host memory";
    return GRT_ENOMEM;
  }
  c->pb = *pb;
  c->device = device;
  c->base = w;
  if ((e = cudaSetDevice(device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess) {
    g_create_error = std::string("CUDA set-up failed: ") + cudaGetErrorString(e);
    delete c;
    return GRT_EDEVICE;
  }
  *out = c;
  return GRT_OK;
}

void grt_destroy(grt_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->solve_plan) {
    ctx->solve_plan->release();
    delete ctx->solve_plan;
  }
  ctx->dx.release();
  ctx->dt.release();
  ctx->du.release();
  ctx->dcoef.release();
  ctx->dse.release();
  ctx->dstatus.release();
  ctx->pdd_scratch.release();
  ctx->plain_part.release();
  ctx->plain_ticket.release();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *grt_last_error(const grt_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int grt_solve(grt_ctx *c, int64_t n, const double *x, const double *t, const uint64_t *ntrees, int K, int L, int M,
              uint64_t seed, uint64_t point_base, double *u_out, double *coef_out, double *se_out,
              int32_t *status_out) {
  if (!c) return GRT_EINVAL;
  if (n < 0) return c->set_error(GRT_EINVAL, "n must be >= 0");
  if (n == 0) return GRT_OK;
  if (!x || !t || !ntrees || !u_out) return c->set_error(GRT_EINVAL, "x, t, ntrees and u_out must be non-NULL");
  if (point_base + (uint64_t)n - 1 > 0xFFFFFFFFull) return c->set_error(GRT_EINVAL, "point_base + n exceeds 2^32");
  const int dim = c->pb.dim;
  for (int64_t i = 0; i < n; ++i) {
    if (!(is_finite(t[i]) && t[i] >= 0.0)) return c->set_error(GRT_EINVAL, "t must be finite and >= 0");
    for (int d = 0; d < dim; ++d)
      if (!is_finite(x[i * dim + d])) return c->set_error(GRT_EINVAL, "x must be finite");
  }
  if (!c->solve_plan) {
    c->solve_plan = new (std::nothrow) grt_plan();
    if (!c->solve_plan) return c->set_error(GRT_ENOMEM, "out of host memory");
    c->solve_plan->ctx = c;
  }
  if (c->solve_plan->cfg.tile != c->solve_cfg.tile) {  // other queue chunks: lay the solve out again
    c->solve_plan->n = -1;
    c->solve_plan->host_ntrees.clear();
  }
  c->solve_plan->cfg = c->solve_cfg;
  int rc = plan_configure(c->solve_plan, n, ntrees, K, L, M);
  if (rc != GRT_OK) return rc;
  GRT_CUDA(c, c->dx.ensure((size_t)n * dim * sizeof(double)));
  GRT_CUDA(c, c->dt.ensure((size_t)n * sizeof(double)));
  GRT_CUDA(c, c->du.ensure((size_t)n * sizeof(double)));
  if (coef_out) GRT_CUDA(c, c->dcoef.ensure((size_t)n * (K + 1) * sizeof(double)));
  if (se_out) GRT_CUDA(c, c->dse.ensure((size_t)n * (K + 1) * sizeof(double)));
  if (status_out) GRT_CUDA(c, c->dstatus.ensure((size_t)n * sizeof(int32_t)));
  cudaStream_t s = c->stream;
  GRT_CUDA(c, cudaMemcpyAsync(c->dx.ptr, x, (size_t)n * dim * sizeof(double), cudaMemcpyHostToDevice, s));
  GRT_CUDA(c, cudaMemcpyAsync(c->dt.ptr, t, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
  rc = plan_execute(c->solve_plan, c->dx.as<double>(), c->dt.as<double>(), seed, point_base, c->du.as<double>(),
                    coef_out ? c->dcoef.as<double>() : nullptr, se_out ? c->dse.as<double>() : nullptr,
                    status_out ? c->dstatus.as<int32_t>() : nullptr, s);
  if (rc != GRT_OK) return rc;
  GRT_CUDA(c, cudaMemcpyAsync(u_out, c->du.ptr, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (coef_out)
    GRT_CUDA(c, cudaMemcpyAsync(coef_out, c->dcoef.ptr, (size_t)n * (K + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (se_out)
    GRT_CUDA(c, cudaMemcpyAsync(se_out, c->dse.ptr, (size_t)n * (K + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (status_out)
    GRT_CUDA(c, cudaMemcpyAsync(status_out, c->dstatus.ptr, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GRT_CUDA(c, cudaStreamSynchronize(s));
  return GRT_OK;
}

int grt_solve_plain(grt_ctx *c, int64_t n, const double *x, const double *t, const uint64_t *ntrees, int K, int L,
                    int M, uint64_t seed, uint64_t point_base, double *u_out, double *coef_out, double *se_out,
                    int32_t *status_out) {
  if (!c) return GRT_EINVAL;
  if (n < 0 || n > 0x7FFFFFFFll) return c->set_error(GRT_EINVAL, "n must be in [0, 2^31)");
  if (K < 0 || K > GRT_MAX_K) return c->set_error(GRT_EINVAL, "K must be in [0, 16]");
  if (L < 0 || M < 0 || L + M > K) return c->set_error(GRT_EINVAL, "need L, M >= 0 and L + M <= K");
  if (n == 0) return GRT_OK;
  if (!x || !t || !ntrees || !u_out) return c->set_error(GRT_EINVAL, "x, t, ntrees and u_out must be non-NULL");
  if (point_base + (uint64_t)n - 1 > 0xFFFFFFFFull) return c->set_error(GRT_EINVAL, "point_base + n exceeds 2^32");
  const int dim = c->pb.dim;
  for (int64_t i = 0; i < n; ++i) {
    if (!(is_finite(t[i]) && t[i] >= 0.0)) return c->set_error(GRT_EINVAL, "t must be finite and >= 0");
    if (ntrees[i] > GRT_MAX_TREES_PER_POINT) return c->set_error(GRT_EINVAL, "ntrees[i] above 2^31 - 1");
    for (int d = 0; d < dim; ++d)
      if (!is_finite(x[i * dim + d])) return c->set_error(GRT_EINVAL, "x must be finite");
  }
  GRT_CUDA(c, cudaSetDevice(c->device));
  // one launch per point, one thread per tree up to the grid's size (then each thread walks several)
  const uint64_t max_blocks = 8ull * (uint64_t)c->num_sms;
  auto blocks_of = [&](uint64_t N) {
    const uint64_t b = (N + grt::kPlainThreads - 1) / grt::kPlainThreads;
    return (unsigned)(b < 1 ? 1 : (b > max_blocks ? max_blocks : b));
  };
  uint64_t most = 1;
  for (int64_t i = 0; i < n; ++i) most = std::max<uint64_t>(most, blocks_of(ntrees[i]));
  GRT_CUDA(c, c->plain_part.ensure((size_t)most * 3 * (K + 2) * sizeof(double)));
  GRT_CUDA(c, c->plain_ticket.ensure((size_t)n * sizeof(uint32_t)));
  GRT_CUDA(c, c->du.ensure((size_t)n * sizeof(double)));
  if (coef_out) GRT_CUDA(c, c->dcoef.ensure((size_t)n * (K + 1) * sizeof(double)));
  if (se_out) GRT_CUDA(c, c->dse.ensure((size_t)n * (K + 1) * sizeof(double)));
  if (status_out) GRT_CUDA(c, c->dstatus.ensure((size_t)n * sizeof(int32_t)));
  cudaStream_t s = c->stream;
  GRT_CUDA(c, cudaMemsetAsync(c->plain_ticket.ptr, 0, (size_t)n * sizeof(uint32_t), s));
  grt::WalkParams w = c->base;
  set_round_keys(w, seed);
  w.K = K;
  for (int64_t i = 0; i < n; ++i) {
    grt::PlainPoint q{};
    for (int d = 0; d < dim; ++d) q.x[d] = x[i * dim + d];
    q.t = t[i];
    q.point = (uint32_t)(point_base + (uint64_t)i);
    q.ntrees = (uint32_t)ntrees[i];
    q.K = K;
    q.L = L;
    q.M = M;
    q.part = c->plain_part.as<double>();
    q.ticket = c->plain_ticket.as<uint32_t>() + i;
    q.u = c->du.as<double>() + i;
    q.coef = coef_out ? c->dcoef.as<double>() + (size_t)i * (K + 1) : nullptr;
    q.se = se_out ? c->dse.as<double>() + (size_t)i * (K + 1) : nullptr;
    q.status = status_out ? c->dstatus.as<int32_t>() + i : nullptr;
    GRT_CUDA(c, grt::launch_plain(dim, c->pb.strategy, w, q, blocks_of(ntrees[i]), s));
  }
  GRT_CUDA(c, cudaMemcpyAsync(u_out, c->du.ptr, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (coef_out)
    GRT_CUDA(c, cudaMemcpyAsync(coef_out, c->dcoef.ptr, (size_t)n * (K + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (se_out)
    GRT_CUDA(c, cudaMemcpyAsync(se_out, c->dse.ptr, (size_t)n * (K + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (status_out)
    GRT_CUDA(c, cudaMemcpyAsync(status_out, c->dstatus.ptr, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GRT_CUDA(c, cudaStreamSynchronize(s));
  return GRT_OK;
}

int grt_plan_create(grt_ctx *c, int64_t n, const uint64_t *ntrees, int K, int L, int M, grt_plan **out) {
  if (!c || !out) return GRT_EINVAL;
  *out = nullptr;
  grt_plan *p = new (std::nothrow) grt_plan();
  if (!p) return c->set_error(GRT_ENOMEM, "out of host memory");
  p->ctx = c;
  p->n = -1;
  int rc = plan_configure(p, n, ntrees, K, L, M);
  if (rc != GRT_OK) {
    p->release();
    delete p;
    return rc;
  }
  *out = p;
  return GRT_OK;
}

int grt_plan_execute(grt_plan *p, const double *d_x, const double *d_t, uint64_t seed, uint64_t point_base,
                     double *d_u, double *d_coef, double *d_se, int32_t *d_status, void *stream) {
  if (!p) return GRT_EINVAL;
  return plan_execute(p, d_x, d_t, seed, point_base, d_u, d_coef, d_se, d_status, (cudaStream_t)stream);
}

int grt_plan_counters(grt_plan *p, uint64_t *nodes, uint64_t *splits, uint64_t *pruned) {
  if (!p) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  unsigned long long st[3] = {0, 0, 0};
  if (p->n > 0) {
    GRT_CUDA(c, cudaSetDevice(c->device));
    GRT_CUDA(c, cudaStreamSynchronize(p->last_stream));
    GRT_CUDA(c, cudaMemcpy(st, p->work.as<unsigned char>() + 8, sizeof(st), cudaMemcpyDeviceToHost));
  }
  if (nodes) *nodes = st[0];
  if (splits) *splits = st[1];
  if (pruned) *pruned = st[2];
  return GRT_OK;
}

int grt_plan_set_timing(grt_plan *p, int on) {
  if (!p) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  if (on) {
    GRT_CUDA(c, cudaSetDevice(c->device));
    for (auto &e : p->ev)
      if (!e) GRT_CUDA(c, cudaEventCreate(&e));
  }
  p->timing = on != 0;
  return GRT_OK;
}

int grt_plan_timing(grt_plan *p, float *walk_ms, float *finalize_ms) {
  if (!p) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  if (!p->timed_last) return c->set_error(GRT_EINVAL, "timing was not enabled for the last execution");
  GRT_CUDA(c, cudaSetDevice(c->device));
  GRT_CUDA(c, cudaEventSynchronize(p->ev[2]));
  float a = 0.f, b = 0.f;
  GRT_CUDA(c, cudaEventElapsedTime(&a, p->ev[0], p->ev[1]));
  GRT_CUDA(c, cudaEventElapsedTime(&b, p->ev[1], p->ev[2]));
  if (walk_ms) *walk_ms = a;
  if (finalize_ms) *finalize_ms = b;
  return GRT_OK;
}

int grt_plan_launches(const grt_plan *p) { return p ? p->launches : 0; }

int grt_set_solve_config(grt_ctx *c, const int32_t *cfg) {
  if (!c || !cfg) return GRT_EINVAL;
  if ((cfg[0] != 4 && cfg[0] != 8) || (cfg[1] != 0 && cfg[1] != 3) || cfg[2] < 0 || cfg[3] < 32 ||
      cfg[3] > (1 << 20) || (cfg[3] & 31))
    return c->set_error(GRT_EINVAL, "config: warps 4|8, smem_levels 0|3, blocks_per_sm >= 0, tile a multiple of 32");
  c->solve_cfg.warps = cfg[0];
  c->solve_cfg.smem_levels = cfg[1];
  c->solve_cfg.blocks_per_sm = cfg[2];
  c->solve_cfg.tile = (uint32_t)cfg[3];
  return GRT_OK;
}

int grt_plan_set_config(grt_plan *p, const int32_t *cfg) {
  if (!p || !cfg) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  if ((cfg[0] != 4 && cfg[0] != 8) || (cfg[1] != 0 && cfg[1] != 3) || cfg[2] < 0 || cfg[3] < 32 ||
      cfg[3] > (1 << 20) || (cfg[3] & 31))
    return c->set_error(GRT_EINVAL, "config: warps 4|8, smem_levels 0|3, blocks_per_sm >= 0, tile a multiple of 32");
  if (p->n < 0) return c->set_error(GRT_EINVAL, "plan has no valid layout");
  grt::WalkConfig nc;
  nc.warps = cfg[0];
  nc.smem_levels = cfg[1];
  nc.blocks_per_sm = cfg[2];
  nc.tile = (uint32_t)cfg[3];
  if (nc.tile != p->cfg.tile) {  // the queue chunks change: lay the plan out again
    const std::vector<uint64_t> nt = p->host_ntrees;
    const grt::WalkConfig old = p->cfg;
    p->cfg = nc;
    p->n = -1;
    const int rc = plan_configure(p, (int64_t)nt.size(), nt.data(), p->K, p->L, p->M);
    if (rc != GRT_OK) {
      p->cfg = old;
      return rc;
    }
  }
  p->cfg = nc;
  return GRT_OK;
}

int grt_plan_get_config(const grt_plan *p, int32_t *cfg) {
  if (!p || !cfg) return GRT_EINVAL;
  cfg[0] = p->cfg.warps;
  cfg[1] = p->cfg.smem_levels;
  cfg[2] = p->cfg.blocks_per_sm;
  cfg[3] = (int32_t)p->cfg.tile;
  return GRT_OK;
}

int grt_plan_autotune(grt_plan *p, const double *d_x, const double *d_t, uint64_t seed, uint64_t point_base,
                      double *d_u, double *d_coef, double *d_se, int32_t *d_status, void *stream, int32_t *cfg_out) {
  if (!p) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  if (p->n <= 0 || c->pb.precision == GRT_FP64) {  // nothing to time / the FP64 walk has one launch shape  // the FP64 walk has one launch shape
    if (cfg_out) grt_plan_get_config(p, cfg_out);
    return GRT_OK;
  }
  GRT_CUDA(c, cudaSetDevice(c->device));
  const bool had_timing = p->timing;
  int rc = grt_plan_set_timing(p, 1);
  if (rc != GRT_OK) return rc;
  static const int32_t cand[][4] = {{4, 0, 0, 512},  {4, 3, 0, 512},  {8, 0, 0, 512},  {8, 3, 0, 512},
                                    {4, 0, 0, 2048}, {4, 3, 0, 2048}, {8, 0, 0, 2048}, {8, 3, 0, 2048},
                                    {4, 0, 4, 512},  {4, 3, 8, 512}};
  int32_t best[4];
  grt_plan_get_config(p, best);
  float best_ms = 1e30f;
  for (const auto &cf : cand) {
    if ((rc = grt_plan_set_config(p, cf)) != GRT_OK) break;
    float wm = 0.f, fm = 0.f, tot = 0.f;
    for (int rep = 0; rep < 3 && rc == GRT_OK; ++rep) {  // first run warms the variant up
      rc = grt_plan_execute(p, d_x, d_t, seed, point_base, d_u, d_coef, d_se, d_status, stream);
      if (rc == GRT_OK) rc = grt_plan_timing(p, &wm, &fm);
      if (rep > 0) tot += wm;
    }
    if (rc != GRT_OK) break;
    if (tot < best_ms) {
      best_ms = tot;
      std::memcpy(best, cf, sizeof(best));
    }
  }
  const int rc2 = grt_plan_set_config(p, best);
  grt_plan_set_timing(p, had_timing ? 1 : 0);
  if (rc != GRT_OK) return rc;
  if (rc2 != GRT_OK) return rc2;
  if (cfg_out) std::memcpy(cfg_out, best, sizeof(best));
  return GRT_OK;
}

int grt_plan_graph_capture(grt_plan *p, const double *d_x, const double *d_t, uint64_t seed, uint64_t point_base,
                           double *d_u, double *d_coef, double *d_se, int32_t *d_status) {
  if (!p) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  if (p->n < 0) return c->set_error(GRT_EINVAL, "plan has no valid layout");
  GRT_CUDA(c, cudaSetDevice(c->device));
  // one plain execution first: kernels and their attributes are loaded outside the capture
  int rc = plan_execute(p, d_x, d_t, seed, point_base, d_u, d_coef, d_se, d_status, c->stream);
  if (rc != GRT_OK) return rc;
  GRT_CUDA(c, cudaStreamSynchronize(c->stream));
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->graph_exec = nullptr;
  p->graph = nullptr;
  GRT_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  rc = plan_execute(p, d_x, d_t, seed, point_base, d_u, d_coef, d_se, d_status, c->stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc != GRT_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return c->cuda_error(e, "cudaStreamEndCapture");
  p->graph = g;
  GRT_CUDA(c, cudaGraphInstantiate(&p->graph_exec, g, 0));
  return GRT_OK;
}

int grt_plan_graph_launch(grt_plan *p, void *stream) {
  if (!p) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  if (!p->graph_exec) return c->set_error(GRT_EINVAL, "no captured graph on this plan");
  GRT_CUDA(c, cudaSetDevice(c->device));
  GRT_CUDA(c, cudaGraphLaunch(p->graph_exec, (cudaStream_t)stream));
  p->last_stream = (cudaStream_t)stream;
  p->timed_last = p->timing;
  p->executed = true;
  return GRT_OK;
}

void grt_plan_destroy(grt_plan *p) {
  if (!p) return;
  cudaSetDevice(p->ctx->device);
  p->release();
  delete p;
}

int grt_plan_kappa(grt_plan *p, double *d_kappa, void *stream) {
  if (!p) return GRT_EINVAL;
  grt_ctx *c = p->ctx;
  if (p->n < 0) return c->set_error(GRT_EINVAL, "plan has no valid layout");
  if (p->n == 0) return GRT_OK;
  if (!d_kappa) return c->set_error(GRT_EINVAL, "kappa must be non-NULL");
  if (!p->executed) return c->set_error(GRT_EINVAL, "the plan has not been executed");
  GRT_CUDA(c, cudaSetDevice(c->device));
  GRT_CUDA(c, grt::launch_kappa((int)p->n, p->K, p->chunk_prefix.as<uint32_t>(), p->ntrees.as<uint32_t>(),
                                p->part.as<double>(), d_kappa, (cudaStream_t)stream));
  return GRT_OK;
}

int grt_pade_error(grt_ctx *c, int64_t n, int K, int L, int M, const double *d_coef, const double *d_se,
                   double *d_err, void *stream) {
  if (!c) return GRT_EINVAL;
  if (n < 0 || n > 0x7FFFFFFFll) return c->set_error(GRT_EINVAL, "n must be in [0, 2^31)");
  if (K < 0 || K > GRT_MAX_K || L < 0 || M < 0 || L + M > K)
    return c->set_error(GRT_EINVAL, "need 0 <= K <= 16, L, M >= 0, L + M <= K");
  if (n == 0) return GRT_OK;
  if (!d_coef || !d_se || !d_err) return c->set_error(GRT_EINVAL, "coef, se and err must be non-NULL");
  GRT_CUDA(c, cudaSetDevice(c->device));
  GRT_CUDA(c, grt::launch_pade_error((int)n, K, L, M, d_coef, d_se, d_err, (cudaStream_t)stream));
  return GRT_OK;
}

int grt_pade(grt_ctx *c, int64_t n, int K, int L, int M, const double *coef, double *u_out, int32_t *status_out) {
  if (!c) return GRT_EINVAL;
  if (n < 0 || n > 0x7FFFFFFFll) return c->set_error(GRT_EINVAL, "n must be in [0, 2^31)");
  if (K < 0 || K > GRT_MAX_K || L < 0 || M < 0 || L + M > K)
    return c->set_error(GRT_EINVAL, "need 0 <= K <= 16, L, M >= 0, L + M <= K");
  if (n == 0) return GRT_OK;
  if (!coef || !u_out) return c->set_error(GRT_EINVAL, "coef and u_out must be non-NULL");
  GRT_CUDA(c, cudaSetDevice(c->device));
  grt::DevBuf dc, du, ds;
  auto cleanup = [&]() {
    dc.release();
    du.release();
    ds.release();
  };
  cudaError_t e;
  if ((e = dc.ensure((size_t)n * (K + 1) * 8)) != cudaSuccess || (e = du.ensure((size_t)n * 8)) != cudaSuccess ||
      (e = ds.ensure((size_t)n * 4)) != cudaSuccess) {
    cleanup();
    return c->cuda_error(e, "grt_pade alloc");
  }
  cudaStream_t s = c->stream;
  if ((e = cudaMemcpyAsync(dc.ptr, coef, (size_t)n * (K + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = grt::launch_pade((int)n, K, L, M, dc.as<double>(), du.as<double>(), ds.as<int32_t>(), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(u_out, du.ptr, (size_t)n * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (status_out && (e = cudaMemcpyAsync(status_out, ds.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    cleanup();
    return c->cuda_error(e, "grt_pade");
  }
  cleanup();
  return GRT_OK;
}

int grt_trees(grt_ctx *c, const double *x, double t, uint64_t point_index, uint64_t first_tree, uint64_t ntrees, int K,
              uint64_t seed, int32_t *order, double *w, uint32_t *nodes, uint64_t *hash) {
  if (!c) return GRT_EINVAL;
  if (!x) return c->set_error(GRT_EINVAL, "x is NULL");
  if (K < 0 || K > GRT_MAX_K) return c->set_error(GRT_EINVAL, "K must be in [0, 16]");
  if (!(is_finite(t) && t >= 0.0)) return c->set_error(GRT_EINVAL, "t must be finite and >= 0");
  for (int d = 0; d < c->pb.dim; ++d)
    if (!is_finite(x[d])) return c->set_error(GRT_EINVAL, "x must be finite");
  if (point_index > 0xFFFFFFFFull || first_tree + ntrees > 0x80000000ull)
    return c->set_error(GRT_EINVAL, "point_index must be < 2^32 and first_tree + ntrees <= 2^31");
  if (ntrees == 0) return GRT_OK;
  GRT_CUDA(c, cudaSetDevice(c->device));
  grt::WalkParams p = c->base;
  set_round_keys(p, seed);
  p.K = K;
  double x0[3] = {0, 0, 0};
  for (int d = 0; d < c->pb.dim; ++d) x0[d] = x[d];
  grt::DevBuf bo, bw, bn, bh;
  auto cleanup = [&]() {
    bo.release();
    bw.release();
    bn.release();
    bh.release();
  };
  cudaError_t e;
  if ((e = bo.ensure(ntrees * 4)) != cudaSuccess || (e = bw.ensure(ntrees * 8)) != cudaSuccess ||
      (e = bn.ensure(ntrees * 4)) != cudaSuccess || (e = bh.ensure(ntrees * 8)) != cudaSuccess) {
    cleanup();
    return c->cuda_error(e, "grt_trees alloc");
  }
  cudaStream_t s = c->stream;
  if ((e = grt::launch_trees(c->pb.precision == GRT_FP64, c->pb.dim, c->pb.strategy, p, x0, t, (uint32_t)point_index,
                             (uint32_t)first_tree, (uint32_t)ntrees, bo.as<int32_t>(), bw.as<double>(),
                             bn.as<uint32_t>(), bh.as<uint64_t>(), s)) != cudaSuccess ||
      (order && (e = cudaMemcpyAsync(order, bo.ptr, ntrees * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (w && (e = cudaMemcpyAsync(w, bw.ptr, ntrees * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (nodes && (e = cudaMemcpyAsync(nodes, bn.ptr, ntrees * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (hash && (e = cudaMemcpyAsync(hash, bh.ptr, ntrees * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    cleanup();
    return c->cuda_error(e, "grt_trees");
  }
  cleanup();
  return GRT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve without any device allocation (grt_solve_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a solve:
// an application whose own pool allocator has reserved the device memory (a
// framework's caching allocator holding the GPU, a host that grants each
// library a fixed share), or code on a latency-critical path where a
// cudaMalloc, which may synchronise the device, is not acceptable.  For them
// the whole work area of a solve lives in one fixed-size array of device
// memory that belongs to the library (every GPU that loads it holds the array
// until the process exits).  The array is shared by every call, so calls whose
// GPU work overlaps in time race on it.  The host-side layout of a call is
// built in file-scope arrays (not on the caller's stack, which may be small)
// under one mutex held until the call has enqueued its copies.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocWorkBytes = 64 + (size_t)GRT_NOALLOC_MAX_POINTS * sizeof(uint32_t);
constexpr size_t kNoAllocMaxChunks =
    (size_t)GRT_NOALLOC_MAX_POINTS + (size_t)GRT_NOALLOC_MAX_TREES / grt::kBinChunk;

constexpr size_t na_align(size_t v) { return (v + 255) & ~(size_t)255; }
// byte offsets of the pieces of the work area
constexpr size_t kNaWork = 0;
constexpr size_t kNaPrefix = na_align(kNaWork + kNoAllocWorkBytes);
constexpr size_t kNaTreePrefix = na_align(kNaPrefix + (GRT_NOALLOC_MAX_POINTS + 1) * sizeof(uint32_t));
constexpr size_t kNaNtrees = na_align(kNaTreePrefix + (GRT_NOALLOC_MAX_POINTS + 1) * sizeof(unsigned long long));
constexpr size_t kNaChunkPrefix = na_align(kNaNtrees + GRT_NOALLOC_MAX_POINTS * sizeof(uint32_t));
constexpr size_t kNaRecO = na_align(kNaChunkPrefix + (GRT_NOALLOC_MAX_POINTS + 1) * sizeof(uint32_t));
constexpr size_t kNaRecSlots = (size_t)GRT_NOALLOC_MAX_TREES + 4 * (size_t)GRT_NOALLOC_MAX_POINTS;  // 4-aligned
constexpr size_t kNaRecW = na_align(kNaRecO + kNaRecSlots);
constexpr size_t kNaPart = na_align(kNaRecW + kNaRecSlots * sizeof(double));
constexpr size_t kNaBytes = na_align(kNaPart + kNoAllocMaxChunks * 4 * (GRT_MAX_K + 2) * sizeof(double));

// The library's fixed work area (about 7 MB).  Host code must not use this
// name as an address: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNaMaxDevices] = {};
// the host-side work layout of the call in progress (guarded by g_noalloc_mutex); the
// host-to-device copies below read these pageable arrays before cudaMemcpyAsync returns
uint32_t g_na_prefix[GRT_NOALLOC_MAX_POINTS + 1], g_na_nt32[GRT_NOALLOC_MAX_POINTS],
    g_na_cprefix[GRT_NOALLOC_MAX_POINTS + 1];
unsigned long long g_na_tprefix[GRT_NOALLOC_MAX_POINTS + 1];

// Device address of the work area on the current device `dev`, looked up once
// per device (on the first call of grt_solve_noalloc on that device).  The
// caller holds g_noalloc_mutex.
cudaError_t noalloc_scratch(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  if (!g_noalloc_ptr[dev]) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
  return cudaSuccess;
}

}  // namespace

extern "C" int grt_solve_noalloc(grt_ctx *c, int64_t n, const double *d_x, const double *d_t, const uint64_t *ntrees,
                                 int K, int L, int M, uint64_t seed, uint64_t point_base, double *d_u, double *d_coef,
                                 double *d_se, int32_t *d_status, void *stream_handle) {
  if (!c) return GRT_EINVAL;
  if (n < 0) return c->set_error(GRT_EINVAL, "n must be >= 0");
  if (n > GRT_NOALLOC_MAX_POINTS)
    return c->set_error(GRT_EINVAL, "grt_solve_noalloc: n above GRT_NOALLOC_MAX_POINTS (4096)");
  if (K < 0 || K > GRT_MAX_K) return c->set_error(GRT_EINVAL, "K must be in [0, 16]");
  if (L < 0 || M < 0 || L + M > K) return c->set_error(GRT_EINVAL, "need L, M >= 0 and L + M <= K");
  if (n == 0) return GRT_OK;
  if (!ntrees || !d_x || !d_t || !d_u) return c->set_error(GRT_EINVAL, "x, t, ntrees and u must be non-NULL");
  if (point_base + (uint64_t)n - 1 > 0xFFFFFFFFull) return c->set_error(GRT_EINVAL, "point_base + n exceeds 2^32");
  // work layout on the host, in the library's fixed arrays (no heap, nothing on the caller's stack)
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  uint32_t *prefix = g_na_prefix, *nt32 = g_na_nt32, *cprefix = g_na_cprefix;
  unsigned long long *tprefix = g_na_tprefix;
  uint64_t items = 0, trees = 0, chunks = 0, recs = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (ntrees[i] > GRT_MAX_TREES_PER_POINT) return c->set_error(GRT_EINVAL, "ntrees[i] above 2^31 - 1");
    prefix[i] = (uint32_t)items;
    tprefix[i] = recs;
    recs += (ntrees[i] + 3) & ~(uint64_t)3;
    cprefix[i] = (uint32_t)chunks;
    nt32[i] = (uint32_t)ntrees[i];
    items += (ntrees[i] + grt::kTile - 1) / grt::kTile;
    chunks += ntrees[i] == 0 ? 1 : (ntrees[i] + grt::kBinChunk - 1) / grt::kBinChunk;
    trees += ntrees[i];
    if (trees > GRT_NOALLOC_MAX_TREES)
      return c->set_error(GRT_EINVAL, "grt_solve_noalloc: total trees above GRT_NOALLOC_MAX_TREES (524288)");
  }
  prefix[n] = (uint32_t)items;
  tprefix[n] = recs;
  cprefix[n] = (uint32_t)chunks;

  GRT_CUDA(c, cudaSetDevice(c->device));
  unsigned char *base = nullptr;
  GRT_CUDA(c, noalloc_scratch(c->device, &base));
  cudaStream_t stream = (cudaStream_t)stream_handle;
  const size_t nn = (size_t)n;
  GRT_CUDA(c, cudaMemcpyAsync(base + kNaPrefix, prefix, (nn + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
  GRT_CUDA(c, cudaMemcpyAsync(base + kNaTreePrefix, tprefix, (nn + 1) * sizeof(unsigned long long),
                              cudaMemcpyHostToDevice, stream));
  GRT_CUDA(c, cudaMemcpyAsync(base + kNaNtrees, nt32, nn * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
  GRT_CUDA(c, cudaMemcpyAsync(base + kNaChunkPrefix, cprefix, (nn + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice,
                              stream));
  // what must start at zero: queue head, counters, the per-point chunk tickets
  GRT_CUDA(c, cudaMemsetAsync(base + kNaWork, 0, 64 + nn * sizeof(uint32_t), stream));

  grt::WalkParams w = c->base;
  set_round_keys(w, seed);
  w.K = K;
  w.point_base = (uint32_t)point_base;
  w.x = d_x;
  w.t = d_t;
  w.ntrees = reinterpret_cast<const uint32_t *>(base + kNaNtrees);
  w.prefix = reinterpret_cast<const uint32_t *>(base + kNaPrefix);
  w.tree_prefix = reinterpret_cast<const unsigned long long *>(base + kNaTreePrefix);
  w.n = (int)n;
  w.tile = grt::kTile;
  w.total_items = (uint32_t)items;
  w.rec_w = base + kNaRecW;
  w.rec_o = base + kNaRecO;
  w.counter = reinterpret_cast<uint32_t *>(base + kNaWork);
  w.stats = reinterpret_cast<unsigned long long *>(base + kNaWork + 8);
  const bool fp64 = c->pb.precision == GRT_FP64;
  if (items > 0)
    GRT_CUDA(c, grt::launch_walk(fp64, c->pb.dim, c->pb.strategy, w, grt::WalkConfig{}, c->num_sms, stream));
  grt::FinalizeParams f{};
  f.rec_w = w.rec_w;
  f.rec_o = w.rec_o;
  f.tree_prefix = w.tree_prefix;
  f.ntrees = w.ntrees;
  f.chunk_prefix = reinterpret_cast<const uint32_t *>(base + kNaChunkPrefix);
  f.total_chunks = (uint32_t)chunks;
  f.part = reinterpret_cast<double *>(base + kNaPart);
  f.n = (int)n;
  f.K = K;
  f.stats = w.stats;
  GRT_CUDA(c, grt::launch_finalize(fp64, f, stream));
  grt::CompleteParams cp{};
  cp.n = (int)n;
  cp.K = K;
  cp.L = L;
  cp.M = M;
  cp.part = f.part;
  cp.chunk_prefix = f.chunk_prefix;
  cp.ntrees = f.ntrees;
  cp.u = d_u;
  cp.coef = d_coef;
  cp.se = d_se;
  cp.status = d_status;
  GRT_CUDA(c, grt::launch_complete(cp, stream));
  return GRT_OK;
}
