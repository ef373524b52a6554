// grt_server.cu -- continuous-batching point-solve server.
//
// The serving form of the probabilistic part of the PDD (Sec. 3): requests
// (point sets with tree budgets) arrive at any time; a scheduler thread runs
// the GPU in steps.  Each step takes tree ranges from every admitted request
// -- smallest remaining work first, up to a step budget -- groups them by
// problem and series shape, and runs the walk and binning kernels over the
// group in one launch each, so requests that arrive while others run join the
// next step and share its launches.  Each point keeps one resident accumulator
// in device memory between steps -- per order and statistic, the compensated
// sum of its chunk sums so far; since every range a step takes starts on a
// binning-chunk boundary of the point's own tree numbering and a point's
// ranges are walked in tree order, its chunk sums are added in chunk order, as
// in a one-shot solve, and a point's result is the same bits whether it was
// solved alone, in one launch, or over many steps.  Admission is by device
// memory: a request waits until its points' accumulators and result rows fit
// the budget (1436 bytes per point).  The groups of one step run on several
// streams at once (disjoint regions of the step buffers), so the launches of
// different requests overlap on the device.  A cancelled request stops taking
// trees after the current step; each of its unfinished points is completed
// from the chunks binned so far (N_done trees, a multiple of 8192) and marked
// SERIES_PARTIAL -- the estimate of Sec. 2.4 over fewer independent trees.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "grt.h"
#include "grt_device.cuh"
#include "grt_host.h"
#include "grt_launch.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kPartStride = 4 * (GRT_MAX_K + 2);  // doubles per chunk-sum slot of a step
constexpr size_t kAccStride = 2 * kPartStride;       // doubles per resident point accumulator (s, c)
constexpr size_t kOutStride = GRT_MAX_K + 1;         // doubles per coef / se row
// resident bytes per admitted point: its accumulator and its result row (u, status, coef, se)
constexpr size_t kPointBytes = kAccStride * 8 + 8 + 4 + 2 * kOutStride * 8;
constexpr int kStreams = 4;                          // streams the groups of a step run on

// First-fit allocator of row ranges in [0, capacity).
class RowPool {
 public:
  void init(uint64_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
    cap_ = cap;
    used_ = 0;
  }
  bool alloc(uint64_t n, uint64_t *start) {
    if (n == 0) {
      *start = 0;
      return true;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *start = it->first;
        const uint64_t rest = it->second - n, at = it->first + n;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t start, uint64_t n) {
    if (n == 0) return;
    used_ -= n;
    auto it = free_.emplace(start, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t used() const { return used_; }
  uint64_t capacity() const { return cap_; }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t cap_ = 0, used_ = 0;
};

struct Request {
  uint64_t id = 0;
  grt_ctx *ctx = nullptr;
  int64_t n = 0;
  int K = 0, L = 0, M = 0;
  uint64_t seed = 0, point_base = 0;
  std::vector<double> x, t;
  std::vector<uint32_t> N;         // trees per point
  std::vector<uint32_t> done;      // trees walked per point (chunk-aligned until the last range)
  std::vector<uint8_t> complete;   // point finished
  uint64_t row = 0;                // resident row of point 0 (accumulator slot and result row of point i: row + i)
  uint64_t remaining = 0;          // trees not yet walked
  int64_t points_left = 0;
  bool admitted = false, finished = false, cancelled = false;
  uint64_t shared_launches = 0, shared_steps = 0;  // launches / steps that also ran another request's trees
  int error = 0;
  std::string error_text;
  std::vector<double> u, coef, se;
  std::vector<int32_t> status;
  Clock::time_point t_submit, t_finish;
};

// One (point, tree range) of a step.
struct Unit {
  Request *r;
  int64_t i;
  uint32_t first, cnt;
};

}  // namespace

struct grt_server {
  int device = 0;
  int num_sms = 0;
  uint64_t budget = 0, step_trees = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t streams[kStreams] = {};
  grt::DevBuf acc_pool, out_u, out_coef, out_se, out_status;
  RowPool rows;  // resident point rows
  grt::DevBuf rec_w, rec_o, meta, xbuf, work, cmeta, step_part;
  size_t meta_points = 0, part_slots = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> pending;
  std::vector<Request *> active;
  std::map<uint64_t, Request *> reqs;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  std::string err;
  int fatal = 0;
  uint64_t steps = 0, trees_walked = 0, launches = 0, shared_launches = 0, cancelled = 0;

  int set_error(int code, const std::string &m) {
    err = m;
    return code;
  }
  void run();
  int run_step(std::vector<Unit> &units, std::string &why);
  int complete_cancelled(const std::vector<Request *> &reqs, std::string &why);
  void release_buffers();
};

namespace {

// Step buffers of a server whose steps take at most step_trees trees: records (8 + 1 bytes per tree
// slot, 4-aligned per point), per-point arrays of up to 2 mp + 1 entries (a group's arrays hold
// n + 1 entries), coordinates, work counters per group, and the step's chunk sums (a unit of c trees
// makes ceil(c / 8192) chunks, at least one, so a step makes at most step_trees / 8192 + mp).
struct StepSizes {
  size_t mp, meta_bytes, xbuf_bytes, work_bytes, rec_slots, part_slots, step_bytes;
};
StepSizes step_sizes(uint64_t step_trees) {
  StepSizes z;
  z.mp = (size_t)std::min<uint64_t>(1ull << 20, std::max<uint64_t>(4096, step_trees / 256));
  z.meta_bytes = 10 * (2 * z.mp + 1) * sizeof(uint32_t);
  z.xbuf_bytes = 2 * z.mp * (GRT_MAX_DIM + 1) * sizeof(double);
  z.work_bytes = 132 * z.mp + 64;
  z.rec_slots = (size_t)step_trees + 4 * z.mp + 64;
  z.part_slots = (size_t)(step_trees / grt::kBinChunk) + z.mp + 1;
  z.step_bytes = z.rec_slots * 9 + z.meta_bytes + z.xbuf_bytes + z.work_bytes + z.part_slots * kPartStride * 8 +
                 64 * 1024;
  return z;
}

// Per-point launch arrays of one group, laid out in one host block and copied once.
struct GroupMeta {
  std::vector<uint32_t> ntrees, prefix, tree_first, point_id, ntotal, out_slot, chunk_prefix;
  std::vector<unsigned long long> tree_prefix;
  std::vector<double> x, t;
};

}  // namespace

int grt_server::run_step(std::vector<Unit> &units, std::string &why) {
  // group the units by (problem context, K, L, M): one walk + one binning launch per group
  // (one Philox key per launch, so the seed is part of the group key)
  auto key_less = [](const Request *a, const Request *b) {
    if (a->ctx != b->ctx) return a->ctx < b->ctx;
    if (a->K != b->K) return a->K < b->K;
    if (a->L != b->L) return a->L < b->L;
    if (a->M != b->M) return a->M < b->M;
    return a->seed < b->seed;
  };
  std::stable_sort(units.begin(), units.end(), [&](const Unit &a, const Unit &b) { return key_less(a.r, b.r); });
  // every group gets disjoint regions of the step buffers (points, records, chunk sums, work
  // counters), so the groups run concurrently on the server's streams
  const size_t u32n = (2 * meta_points + 1) * sizeof(uint32_t);  // entries of one per-point array
  unsigned char *mb = meta.as<unsigned char>();
  uint32_t *a_ntrees = reinterpret_cast<uint32_t *>(mb + 0 * u32n), *a_prefix = reinterpret_cast<uint32_t *>(mb + 1 * u32n),
           *a_first = reinterpret_cast<uint32_t *>(mb + 2 * u32n), *a_pid = reinterpret_cast<uint32_t *>(mb + 3 * u32n),
           *a_ntot = reinterpret_cast<uint32_t *>(mb + 4 * u32n), *a_oslot = reinterpret_cast<uint32_t *>(mb + 5 * u32n),
           *a_cpre = reinterpret_cast<uint32_t *>(mb + 6 * u32n);
  unsigned long long *a_tpre = reinterpret_cast<unsigned long long *>(mb + 8 * u32n);
  double *a_x = xbuf.as<double>(), *a_t = a_x + 2 * meta_points * GRT_MAX_DIM;
  size_t pt_off = 0, rec_off = 0, work_off = 0, part_off = 0;
  int gidx = 0;
  size_t g0 = 0;
  while (g0 < units.size()) {
    size_t g1 = g0 + 1;
    const Request *r0 = units[g0].r;
    while (g1 < units.size() && !key_less(r0, units[g1].r) && !key_less(units[g1].r, r0)) ++g1;
    grt_ctx *c = r0->ctx;
    const int K = r0->K, dim = c->pb.dim;
    const size_t n = g1 - g0;
    GroupMeta m;
    m.ntrees.resize(n);
    m.prefix.resize(n + 1);
    m.tree_first.resize(n);
    m.point_id.resize(n);
    m.ntotal.resize(n);
    m.out_slot.resize(n);
    m.chunk_prefix.resize(n + 1);
    m.tree_prefix.resize(n + 1);
    m.x.resize(n * dim);
    m.t.resize(n);
    uint64_t items = 0, recs = 0, chunks = 0;
    const Request *last = nullptr;
    int distinct = 0;
    for (size_t k = 0; k < n; ++k) {
      const Unit &u = units[g0 + k];
      const Request &r = *u.r;
      if (u.r != last) {  // units of one request are contiguous within the group
        ++distinct;
        last = u.r;
      }
      m.ntrees[k] = u.cnt;
      m.prefix[k] = (uint32_t)items;
      m.tree_prefix[k] = recs;
      m.chunk_prefix[k] = (uint32_t)chunks;
      m.tree_first[k] = u.first;
      m.point_id[k] = (uint32_t)(r.point_base + (uint64_t)u.i);
      m.ntotal[k] = r.N[u.i];
      m.out_slot[k] = (uint32_t)(r.row + (uint64_t)u.i);
      for (int d = 0; d < dim; ++d) m.x[k * dim + d] = r.x[(size_t)u.i * dim + d];
      m.t[k] = r.t[u.i];
      items += (u.cnt + grt::kTile - 1) / grt::kTile;
      recs += (u.cnt + 3) & ~3u;
      chunks += u.cnt == 0 ? 1 : (u.cnt + grt::kBinChunk - 1) / grt::kBinChunk;
    }
    m.prefix[n] = (uint32_t)items;
    m.tree_prefix[n] = recs;
    m.chunk_prefix[n] = (uint32_t)chunks;
    if (distinct > 1) {  // this walk launch batches trees of several requests
      ++shared_launches;
      last = nullptr;
      for (size_t k = g0; k < g1; ++k)
        if (units[k].r != last) {
          last = units[k].r;
          ++units[k].r->shared_launches;
        }
    }
    const size_t work_bytes = (64 + n * sizeof(uint32_t) + 63) & ~(size_t)63;
    if (pt_off + n + 1 > 2 * meta_points + 1 || (rec_off + recs) * 8 > rec_w.cap ||
        rec_off + recs > rec_o.cap || work_off + work_bytes > work.cap || part_off + chunks > part_slots) {
      why = "step larger than the server's step buffers";
      return GRT_EINVAL;
    }
    cudaStream_t st = streams[gidx % kStreams];
    uint32_t *d_ntrees = a_ntrees + pt_off, *d_prefix = a_prefix + pt_off, *d_first = a_first + pt_off,
             *d_pid = a_pid + pt_off, *d_ntot = a_ntot + pt_off, *d_oslot = a_oslot + pt_off,
             *d_cpre = a_cpre + pt_off;
    double *d_part = step_part.as<double>() + part_off * kPartStride;
    unsigned long long *d_tpre = a_tpre + pt_off;
    double *d_x = a_x + pt_off * GRT_MAX_DIM, *d_t = a_t + pt_off;
    unsigned char *d_work = work.as<unsigned char>() + work_off;
    unsigned char *d_recw = rec_w.as<unsigned char>() + rec_off * 8;  // 8 bytes per slot: FP32 or FP64 records
    uint8_t *d_reco = rec_o.as<uint8_t>() + rec_off;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    cp(d_ntrees, m.ntrees.data(), n * 4);
    cp(d_prefix, m.prefix.data(), (n + 1) * 4);
    cp(d_first, m.tree_first.data(), n * 4);
    cp(d_pid, m.point_id.data(), n * 4);
    cp(d_ntot, m.ntotal.data(), n * 4);
    cp(d_oslot, m.out_slot.data(), n * 4);
    cp(d_cpre, m.chunk_prefix.data(), (n + 1) * 4);
    cp(d_tpre, m.tree_prefix.data(), (n + 1) * 8);
    cp(d_x, m.x.data(), n * dim * 8);
    cp(d_t, m.t.data(), n * 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_work, 0, 64 + n * sizeof(uint32_t), st);
    if (e != cudaSuccess) {
      why = std::string("step copies: ") + cudaGetErrorString(e);
      return GRT_EDEVICE;
    }
    grt::WalkParams w = c->base;
    uint32_t k0 = (uint32_t)r0->seed, k1 = (uint32_t)(r0->seed >> 32);
    for (int r = 0; r < 10; ++r) {
      w.rk0[r] = k0;
      w.rk1[r] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    w.K = K;
    w.point_base = 0;
    w.x = d_x;
    w.t = d_t;
    w.ntrees = d_ntrees;
    w.prefix = d_prefix;
    w.tree_prefix = d_tpre;
    w.tree_first = d_first;
    w.point_id = d_pid;
    w.n = (int)n;
    w.tile = grt::kTile;
    w.total_items = (uint32_t)items;
    w.rec_w = d_recw;
    w.rec_o = d_reco;
    w.counter = reinterpret_cast<uint32_t *>(d_work);
    w.stats = reinterpret_cast<unsigned long long *>(d_work + 8);
    const bool fp64 = c->pb.precision == GRT_FP64;
    if (items > 0) {
      e = grt::launch_walk(fp64, dim, c->pb.strategy, w, grt::WalkConfig{}, num_sms, st);
      ++launches;
    }
    // the group's chunk sums, in the step's chunk-sum buffer at the group's chunk numbering
    grt::FinalizeParams f{};
    f.rec_w = d_recw;
    f.rec_o = d_reco;
    f.tree_prefix = d_tpre;
    f.ntrees = d_ntrees;
    f.chunk_prefix = d_cpre;
    f.total_chunks = (uint32_t)chunks;
    f.part = d_part;
    f.part_stride = kPartStride;
    f.n = (int)n;
    f.K = K;
    f.stats = w.stats;
    if (e == cudaSuccess) e = grt::launch_finalize(fp64, f, st);
    ++launches;
    // each unit's chunk sums into its point's accumulator; points whose last range this is:
    // a_n, SE_n, Pade
    grt::FoldParams fo{};
    fo.n = (int)n;
    fo.K = K;
    fo.L = r0->L;
    fo.M = r0->M;
    fo.part = d_part;
    fo.part_stride = kPartStride;
    fo.chunk_prefix = d_cpre;
    fo.acc = acc_pool.as<double>();
    fo.acc_stride = kAccStride;
    fo.slot = d_oslot;
    fo.tree_first = d_first;
    fo.ntrees = d_ntrees;
    fo.ntotal = d_ntot;
    fo.out_stride = kOutStride;
    fo.u = out_u.as<double>();
    fo.coef = out_coef.as<double>();
    fo.se = out_se.as<double>();
    fo.status = out_status.as<int32_t>();
    if (e == cudaSuccess) e = grt::launch_fold(fo, st);
    ++launches;
    if (e != cudaSuccess) {
      why = std::string("step launch: ") + cudaGetErrorString(e);
      return GRT_EDEVICE;
    }
    pt_off += n + 1;
    rec_off += recs;
    work_off += work_bytes;
    part_off += chunks;
    ++gidx;
    g0 = g1;
  }
  for (int k = 0; k < kStreams && k < std::max(gidx, 1); ++k) {
    const cudaError_t e = cudaStreamSynchronize(streams[k]);
    if (e != cudaSuccess) {
      why = std::string("step: ") + cudaGetErrorString(e);
      return GRT_EDEVICE;
    }
  }
  return GRT_OK;
}

// Completion of the unfinished points of cancelled requests from their accumulators (the chunks
// binned so far: N_done trees, where a point whose first range never ran has zero sums).
int grt_server::complete_cancelled(const std::vector<Request *> &reqs, std::string &why) {
  // one completion launch per series shape (K, L, M); points of one request share it
  std::map<std::tuple<int, int, int>, std::vector<std::pair<Request *, int64_t>>> by_shape;
  for (Request *r : reqs)
    for (int64_t i = 0; i < r->n; ++i)
      if (!r->complete[i]) by_shape[std::make_tuple(r->K, r->L, r->M)].push_back({r, i});
  for (auto &kv : by_shape) {
    const auto &pts = kv.second;
    const size_t n = pts.size();
    std::vector<uint32_t> h((size_t)3 * n);  // slot, trees so far (= N_done), trees of this "range" (none)
    for (size_t k = 0; k < n; ++k) {
      const Request *r = pts[k].first;
      const int64_t i = pts[k].second;
      h[k] = (uint32_t)(r->row + (uint64_t)i);
      h[n + k] = r->done[i];  // an unfinished point's ranges end on chunk boundaries
      h[2 * n + k] = 0u;
    }
    cudaError_t e = cmeta.ensure(h.size() * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cmeta.ptr, h.data(), h.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, streams[0]);
    grt::FoldParams fo{};
    fo.n = (int)n;
    fo.K = std::get<0>(kv.first);
    fo.L = std::get<1>(kv.first);
    fo.M = std::get<2>(kv.first);
    fo.part = nullptr;  // no chunk sums to add: complete from the accumulator with N = N_done
    fo.acc = acc_pool.as<double>();
    fo.acc_stride = kAccStride;
    fo.slot = cmeta.as<uint32_t>();
    fo.tree_first = fo.slot + n;
    fo.ntrees = fo.slot + 2 * n;
    fo.ntotal = fo.tree_first;
    fo.out_stride = kOutStride;
    fo.u = out_u.as<double>();
    fo.coef = out_coef.as<double>();
    fo.se = out_se.as<double>();
    fo.status = out_status.as<int32_t>();
    fo.extra_status = GRT_STATUS_SERIES_PARTIAL;
    if (e == cudaSuccess) e = grt::launch_fold(fo, streams[0]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(streams[0]);
    ++launches;
    if (e != cudaSuccess) {
      why = std::string("completion of cancelled requests: ") + cudaGetErrorString(e);
      return GRT_EDEVICE;
    }
  }
  return GRT_OK;
}

void grt_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lock(mu);
  auto fail_all = [&](int rc, const std::string &why) {
    fatal = rc;
    err = why;
    for (Request *r : active) {
      r->error = rc;
      r->error_text = why;
      r->finished = true;
      r->t_finish = Clock::now();
    }
    active.clear();
    cv_done.notify_all();
  };
  // requests whose every point is done take their results off the device and free their rows
  auto finish_done = [&]() {
    for (size_t k = 0; k < active.size();) {
      Request *r = active[k];
      if (r->points_left > 0) {
        ++k;
        continue;
      }
      const size_t n = (size_t)r->n, K1 = (size_t)r->K + 1;
      r->u.resize(n);
      r->status.resize(n);
      r->coef.resize(n * K1);
      r->se.resize(n * K1);
      cudaError_t e = cudaMemcpy(r->u.data(), out_u.as<double>() + r->row, n * 8, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(r->status.data(), out_status.as<int32_t>() + r->row, n * 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy2D(r->coef.data(), K1 * 8, out_coef.as<double>() + r->row * kOutStride, kOutStride * 8, K1 * 8,
                         n, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy2D(r->se.data(), K1 * 8, out_se.as<double>() + r->row * kOutStride, kOutStride * 8, K1 * 8, n,
                         cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        r->error = GRT_EDEVICE;
        r->error_text = cudaGetErrorString(e);
      }
      rows.release(r->row, (uint64_t)r->n);
      r->finished = true;
      r->t_finish = Clock::now();
      active.erase(active.begin() + (ptrdiff_t)k);
    }
    cv_done.notify_all();
  };
  while (!stop) {
    // admission: first come, first admitted, while the resident state fits the budget
    while (!pending.empty()) {
      Request *r = pending.front();
      uint64_t row = 0;
      if (!rows.alloc((uint64_t)r->n, &row)) break;
      r->row = row;
      r->admitted = true;
      pending.pop_front();
      active.push_back(r);
    }
    // cancelled requests: their unfinished points are completed from the trees binned so far
    std::vector<Request *> canc;
    for (Request *r : active)
      if (r->cancelled && r->points_left > 0) canc.push_back(r);
    if (!canc.empty()) {
      lock.unlock();
      std::string why;
      const int rc = complete_cancelled(canc, why);
      lock.lock();
      if (rc != GRT_OK) {
        fail_all(rc, why);
        continue;
      }
      for (Request *r : canc) {
        for (int64_t i = 0; i < r->n; ++i) r->complete[i] = 1;
        r->points_left = 0;
        ++cancelled;
      }
      finish_done();
      continue;
    }
    if (active.empty()) {
      cv_work.wait(lock);
      continue;
    }
    // the step's work: smallest remaining first; ranges start on chunk boundaries
    std::vector<Request *> order(active);
    std::stable_sort(order.begin(), order.end(), [](const Request *a, const Request *b) {
      if (a->remaining != b->remaining) return a->remaining < b->remaining;
      return a->id < b->id;
    });
    std::vector<Unit> units;
    uint64_t budget_left = step_trees;
    for (Request *r : order) {
      if (r->cancelled) continue;
      for (int64_t i = 0; i < r->n && units.size() < meta_points; ++i) {
        if (r->complete[i]) continue;
        const uint32_t left = r->N[i] - r->done[i];
        uint64_t take = std::min<uint64_t>(left, budget_left);
        if (take < left) take -= take % grt::kBinChunk;  // a partial range ends on a chunk boundary
        if (take == 0 && left > 0) continue;
        units.push_back(Unit{r, i, r->done[i], (uint32_t)take});
        budget_left -= take;
        if (budget_left < grt::kBinChunk) budget_left = 0;
      }
      if (budget_left == 0 || units.size() >= meta_points) break;
    }
    if (units.empty()) {  // only cancelled requests are left: the next pass completes them
      cv_work.wait_for(lock, std::chrono::milliseconds(1));
      continue;
    }
    lock.unlock();
    std::string why;
    const int rc = run_step(units, why);
    lock.lock();
    ++steps;
    if (rc != GRT_OK) {
      fail_all(rc, why);
      continue;
    }
    // bookkeeping
    std::vector<Request *> in_step;
    for (const Unit &u : units) {
      Request *r = u.r;
      if (in_step.empty() || in_step.back() != r) in_step.push_back(r);
      r->done[u.i] += u.cnt;
      r->remaining -= u.cnt;
      trees_walked += u.cnt;
      if (r->done[u.i] == r->N[u.i]) {
        r->complete[u.i] = 1;
        --r->points_left;
      }
    }
    std::sort(in_step.begin(), in_step.end());
    in_step.erase(std::unique(in_step.begin(), in_step.end()), in_step.end());
    if (in_step.size() > 1)
      for (Request *r : in_step) ++r->shared_steps;
    finish_done();
  }
}

extern "C" {

void grt_server::release_buffers() {
  acc_pool.release();
  step_part.release();
  out_u.release();
  out_status.release();
  out_coef.release();
  out_se.release();
  rec_w.release();
  rec_o.release();
  meta.release();
  xbuf.release();
  work.release();
  cmeta.release();
  for (auto &st : streams)
    if (st) {
      cudaStreamDestroy(st);
      st = nullptr;
    }
  stream = nullptr;
}

int grt_server_sizes(uint64_t step_trees, uint64_t *step_bytes, uint64_t *point_bytes) {
  if (step_trees == 0) step_trees = 1ull << 27;
  if (step_trees < (uint64_t)grt::kBinChunk || step_trees > (1ull << 31)) return GRT_EINVAL;
  if (step_bytes) *step_bytes = step_sizes(step_trees).step_bytes;
  if (point_bytes) *point_bytes = kPointBytes;
  return GRT_OK;
}

int grt_server_create(int device, uint64_t mem_budget_bytes, uint64_t step_trees, grt_server **out) {
  if (!out) return GRT_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GRT_EDEVICE;
  if (step_trees == 0) step_trees = 1ull << 27;
  if (step_trees < (uint64_t)grt::kBinChunk || step_trees > (1ull << 31)) return GRT_EINVAL;
  grt_server *s = new (std::nothrow) grt_server();
  if (!s) return GRT_ENOMEM;
  s->device = device;
  s->budget = mem_budget_bytes;
  s->step_trees = step_trees;
  const StepSizes z = step_sizes(step_trees);
  s->meta_points = z.mp;
  s->part_slots = z.part_slots;
  if (mem_budget_bytes < z.step_bytes + (1ull << 20)) {
    delete s;
    return GRT_EINVAL;  // the budget must hold the step buffers and some resident state
  }
  const uint64_t cap = std::min<uint64_t>((mem_budget_bytes - z.step_bytes) / kPointBytes, 1ull << 31);  // points
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
  for (int k = 0; k < kStreams && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = s->acc_pool.ensure(cap * kAccStride * 8);
  if (e == cudaSuccess) e = s->out_u.ensure(cap * 8);
  if (e == cudaSuccess) e = s->out_status.ensure(cap * 4);
  if (e == cudaSuccess) e = s->out_coef.ensure(cap * kOutStride * 8);
  if (e == cudaSuccess) e = s->out_se.ensure(cap * kOutStride * 8);
  if (e == cudaSuccess) e = s->rec_w.ensure(z.rec_slots * 8);
  if (e == cudaSuccess) e = s->rec_o.ensure(z.rec_slots);
  if (e == cudaSuccess) e = s->meta.ensure(z.meta_bytes);
  if (e == cudaSuccess) e = s->xbuf.ensure(z.xbuf_bytes);
  if (e == cudaSuccess) e = s->work.ensure(z.work_bytes);
  if (e == cudaSuccess) e = s->step_part.ensure(z.part_slots * kPartStride * 8);
  if (e != cudaSuccess) {
    s->release_buffers();
    delete s;
    return e == cudaErrorMemoryAllocation ? GRT_ENOMEM : GRT_EDEVICE;
  }
  s->stream = s->streams[0];
  s->rows.init(cap);
  s->worker = std::thread([s]() { s->run(); });
  *out = s;
  return GRT_OK;
}

void grt_server_destroy(grt_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->reqs) delete kv.second;
  cudaSetDevice(s->device);
  s->release_buffers();
  delete s;
}

const char *grt_server_last_error(const grt_server *s) { return s ? s->err.c_str() : ""; }

int grt_submit(grt_server *s, grt_ctx *c, int64_t n, const double *x, const double *t, const uint64_t *ntrees, int K,
               int L, int M, uint64_t seed, uint64_t point_base, uint64_t *request_id) {
  if (!s || !c || !request_id) return GRT_EINVAL;
  if (n < 0 || n > 0x7FFFFFFFll) return s->set_error(GRT_EINVAL, "n must be in [0, 2^31)");
  if (K < 0 || K > GRT_MAX_K || L < 0 || M < 0 || L + M > K)
    return s->set_error(GRT_EINVAL, "need 0 <= K <= 16, L, M >= 0, L + M <= K");
  if (c->device != s->device) return s->set_error(GRT_EINVAL, "context and server are on different devices");
  if (n > 0 && (!x || !t || !ntrees)) return s->set_error(GRT_EINVAL, "x, t and ntrees must be non-NULL");
  if (point_base + (uint64_t)(n > 0 ? n - 1 : 0) > 0xFFFFFFFFull)
    return s->set_error(GRT_EINVAL, "point_base + n exceeds 2^32");
  Request *r = new (std::nothrow) Request();
  if (!r) return GRT_ENOMEM;
  const int dim = c->pb.dim;
  r->ctx = c;
  r->n = n;
  r->K = K;
  r->L = L;
  r->M = M;
  r->seed = seed;
  r->point_base = point_base;
  r->x.assign(x, x + n * dim);
  r->t.assign(t, t + n);
  r->N.resize(n);
  r->done.assign(n, 0);
  r->complete.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (ntrees[i] > GRT_MAX_TREES_PER_POINT || !std::isfinite(t[i]) || t[i] < 0.0) {
      delete r;
      return s->set_error(GRT_EINVAL, "ntrees[i] <= 2^31 - 1 and finite t[i] >= 0 required");
    }
    r->N[i] = (uint32_t)ntrees[i];
    r->remaining += ntrees[i];
  }
  r->points_left = n;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fatal) {
      delete r;
      return s->set_error(s->fatal, "server stopped after a device error: " + s->err);
    }
    if ((uint64_t)n > s->rows.capacity()) {
      delete r;
      return s->set_error(GRT_ENOMEM, "request larger than the server's memory budget");
    }
    r->id = s->next_id++;
    if (n == 0) {  // nothing to do
      r->finished = true;
      r->t_finish = r->t_submit;
    } else {
      s->pending.push_back(r);
    }
    s->reqs[r->id] = r;
    *request_id = r->id;
  }
  s->cv_work.notify_all();
  return GRT_OK;
}

int grt_cancel(grt_server *s, uint64_t request_id) {
  if (!s) return GRT_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return s->set_error(GRT_EINVAL, "unknown request id");
    Request *r = it->second;
    if (r->finished || r->cancelled) return GRT_OK;
    r->cancelled = true;
    if (!r->admitted) {  // still queued: no tree was walked, every point ends with N_done = 0
      for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
        if (*p == r) {
          s->pending.erase(p);
          break;
        }
      const size_t n = (size_t)r->n, K1 = (size_t)r->K + 1;
      r->u.assign(n, 0.0);
      r->coef.assign(n * K1, 0.0);
      r->se.assign(n * K1, 0.0);
      // the Pade of an all-zero series: every pivot vanishes, [L/M] falls to [L-M/0] (singular when M > 0)
      r->status.assign(n, GRT_STATUS_SERIES_PARTIAL | (r->M > 0 ? GRT_STATUS_PADE_SINGULAR : 0));
      r->finished = true;
      r->t_finish = Clock::now();
      ++s->cancelled;
      s->cv_done.notify_all();
      return GRT_OK;
    }
  }
  s->cv_work.notify_all();
  return GRT_OK;
}

int grt_poll_ex(grt_server *s, uint64_t request_id, int timeout_ms, double *u_out, double *coef_out, double *se_out,
                int32_t *status_out, uint64_t *ntrees_done, grt_request_info *info) {
  if (!s) return GRT_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return s->set_error(GRT_EINVAL, "unknown request id");
  Request *r = it->second;
  if (!r->finished && timeout_ms != 0) {
    const auto until = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (!r->finished) {
      if (timeout_ms < 0) s->cv_done.wait(lock);
      else if (s->cv_done.wait_until(lock, until) == std::cv_status::timeout) break;
    }
  }
  if (!r->finished) return GRT_EAGAIN;
  const int rc = r->error;
  const size_t n = (size_t)r->n, K1 = (size_t)r->K + 1;
  if (rc == GRT_OK) {
    if (u_out && n) std::memcpy(u_out, r->u.data(), n * 8);
    if (status_out && n) std::memcpy(status_out, r->status.data(), n * 4);
    if (coef_out && n) std::memcpy(coef_out, r->coef.data(), n * K1 * 8);
    if (se_out && n) std::memcpy(se_out, r->se.data(), n * K1 * 8);
    if (ntrees_done)
      for (size_t i = 0; i < n; ++i) ntrees_done[i] = r->done[i];
  } else {
    s->err = r->error_text;
  }
  if (info) {
    info->latency_s = std::chrono::duration<double>(r->t_finish - r->t_submit).count();
    info->shared_launches = r->shared_launches;
    info->shared_steps = r->shared_steps;
    info->cancelled = r->cancelled ? 1 : 0;
  }
  s->reqs.erase(it);
  delete r;
  return rc;
}

int grt_poll(grt_server *s, uint64_t request_id, int timeout_ms, double *u_out, double *coef_out, double *se_out,
             int32_t *status_out, double *latency_s) {
  grt_request_info info{};
  const int rc = grt_poll_ex(s, request_id, timeout_ms, u_out, coef_out, se_out, status_out, nullptr, &info);
  if (rc != GRT_EAGAIN && latency_s) *latency_s = info.latency_s;
  return rc;
}

int grt_server_stats(grt_server *s, uint64_t *steps, uint64_t *trees, uint64_t *launches, uint64_t *resident_bytes,
                     uint64_t *pending_requests, uint64_t *active_requests, uint64_t *shared_launches,
                     uint64_t *cancelled_requests) {
  if (!s) return GRT_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (steps) *steps = s->steps;
  if (trees) *trees = s->trees_walked;
  if (launches) *launches = s->launches;
  if (resident_bytes)
    *resident_bytes = s->rows.used() * kPointBytes;
  if (pending_requests) *pending_requests = s->pending.size();
  if (active_requests) *active_requests = s->active.size();
  if (shared_launches) *shared_launches = s->shared_launches;
  if (cancelled_requests) *cancelled_requests = s->cancelled;
  return GRT_OK;
}

}  // extern "C"
