// grt_server.cu -- continuous-batching point-solve server.
//
// The serving form of the probabilistic part of the PDD (Sec. 3): requests
// (point sets with tree budgets) arrive at any time; a scheduler thread runs
// the GPU in steps.  Each step takes tree ranges from every admitted request
// -- smallest remaining work first, up to a step budget -- groups them by
// problem and series shape, and runs the walk and binning kernels over the
// group in one launch each, so requests that arrive while others run join the
// next step and share its launches.  Per-point chunk sums stay resident in
// device memory between steps; since every range a step takes starts on a
// binning-chunk boundary of the point's own tree numbering and the chunk sums
// are added in chunk order when the point completes, a point's result is the
// same bits whether it was solved alone, in one launch, or over many steps.
// Admission is by device memory: a request waits until its resident chunk
// sums and result rows fit the budget.
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
#include <vector>

#include "grt.h"
#include "grt_device.cuh"
#include "grt_host.h"
#include "grt_launch.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kPartStride = 4 * (GRT_MAX_K + 2);  // doubles per resident chunk slot
constexpr size_t kOutStride = GRT_MAX_K + 1;         // doubles per coef / se row

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
  std::vector<uint32_t> part_slot; // first resident chunk slot per point
  uint64_t part_row = 0, part_rows = 0, out_row = 0;
  uint64_t remaining = 0;          // trees not yet walked
  int64_t points_left = 0;
  bool admitted = false, finished = false;
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

uint32_t point_chunks(uint32_t N) { return N == 0 ? 1u : (N + grt::kBinChunk - 1) / grt::kBinChunk; }

}  // namespace

struct grt_server {
  int device = 0;
  int num_sms = 0;
  uint64_t budget = 0, step_trees = 0;
  cudaStream_t stream = nullptr;
  grt::DevBuf part_pool, out_u, out_coef, out_se, out_status;
  RowPool part_rows, out_rows;
  grt::DevBuf rec_w, rec_o, meta, xbuf, work;
  size_t meta_points = 0;
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
  uint64_t steps = 0, trees_walked = 0, launches = 0;

  int set_error(int code, const std::string &m) {
    err = m;
    return code;
  }
  void run();
  int run_step(std::vector<Unit> &units, std::string &why);
};

namespace {

// Per-point launch arrays of one group, laid out in one host block and copied once.
struct GroupMeta {
  std::vector<uint32_t> ntrees, prefix, tree_first, point_id, ntotal, part_slot, out_slot, chunk_prefix;
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
    m.part_slot.resize(n);
    m.out_slot.resize(n);
    m.chunk_prefix.resize(n + 1);
    m.tree_prefix.resize(n + 1);
    m.x.resize(n * dim);
    m.t.resize(n);
    uint64_t items = 0, recs = 0, chunks = 0;
    for (size_t k = 0; k < n; ++k) {
      const Unit &u = units[g0 + k];
      const Request &r = *u.r;
      m.ntrees[k] = u.cnt;
      m.prefix[k] = (uint32_t)items;
      m.tree_prefix[k] = recs;
      m.chunk_prefix[k] = (uint32_t)chunks;
      m.tree_first[k] = u.first;
      m.point_id[k] = (uint32_t)(r.point_base + (uint64_t)u.i);
      m.ntotal[k] = r.N[u.i];
      m.part_slot[k] = r.part_slot[u.i];
      m.out_slot[k] = (uint32_t)(r.out_row + (uint64_t)u.i);
      for (int d = 0; d < dim; ++d) m.x[k * dim + d] = r.x[(size_t)u.i * dim + d];
      m.t[k] = r.t[u.i];
      items += (u.cnt + grt::kTile - 1) / grt::kTile;
      recs += (u.cnt + 3) & ~3u;
      chunks += u.cnt == 0 ? 1 : (u.cnt + grt::kBinChunk - 1) / grt::kBinChunk;
    }
    m.prefix[n] = (uint32_t)items;
    m.tree_prefix[n] = recs;
    m.chunk_prefix[n] = (uint32_t)chunks;
    // device copies of the group's arrays (the buffers are sized at server creation)
    if (n > meta_points) {
      why = "step has more points than the server's step buffers hold";
      return GRT_EINVAL;
    }
    unsigned char *mb = meta.as<unsigned char>();
    const size_t u32n = (meta_points + 1) * sizeof(uint32_t);
    uint32_t *d_ntrees = reinterpret_cast<uint32_t *>(mb + 0 * u32n), *d_prefix = reinterpret_cast<uint32_t *>(mb + 1 * u32n),
             *d_first = reinterpret_cast<uint32_t *>(mb + 2 * u32n), *d_pid = reinterpret_cast<uint32_t *>(mb + 3 * u32n),
             *d_ntot = reinterpret_cast<uint32_t *>(mb + 4 * u32n), *d_pslot = reinterpret_cast<uint32_t *>(mb + 5 * u32n),
             *d_oslot = reinterpret_cast<uint32_t *>(mb + 6 * u32n), *d_cpre = reinterpret_cast<uint32_t *>(mb + 7 * u32n);
    unsigned long long *d_tpre = reinterpret_cast<unsigned long long *>(mb + 8 * u32n);
    double *d_x = xbuf.as<double>(), *d_t = d_x + meta_points * GRT_MAX_DIM;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
    };
    cp(d_ntrees, m.ntrees.data(), n * 4);
    cp(d_prefix, m.prefix.data(), (n + 1) * 4);
    cp(d_first, m.tree_first.data(), n * 4);
    cp(d_pid, m.point_id.data(), n * 4);
    cp(d_ntot, m.ntotal.data(), n * 4);
    cp(d_pslot, m.part_slot.data(), n * 4);
    cp(d_oslot, m.out_slot.data(), n * 4);
    cp(d_cpre, m.chunk_prefix.data(), (n + 1) * 4);
    cp(d_tpre, m.tree_prefix.data(), (n + 1) * 8);
    cp(d_x, m.x.data(), n * dim * 8);
    cp(d_t, m.t.data(), n * 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(work.ptr, 0, 64 + n * sizeof(uint32_t), stream);
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
    w.rec_w = rec_w.ptr;
    w.rec_o = rec_o.as<uint8_t>();
    w.counter = work.as<uint32_t>();
    w.stats = reinterpret_cast<unsigned long long *>(work.as<unsigned char>() + 8);
    const bool fp64 = c->pb.precision == GRT_FP64;
    if (items > 0) {
      e = grt::launch_walk(fp64, dim, c->pb.strategy, w, grt::WalkConfig{}, num_sms, stream);
      ++launches;
    }
    grt::FinalizeParams f{};
    f.rec_w = rec_w.ptr;
    f.rec_o = rec_o.as<uint8_t>();
    f.tree_prefix = d_tpre;
    f.ntrees = d_ntrees;
    f.chunk_prefix = d_cpre;
    f.total_chunks = (uint32_t)chunks;
    f.part = part_pool.as<double>();
    f.done = reinterpret_cast<uint32_t *>(work.as<unsigned char>() + 64);
    f.tree_first = d_first;
    f.ntotal = d_ntot;
    f.part_slot = d_pslot;
    f.out_slot = d_oslot;
    f.part_stride = kPartStride;
    f.out_stride = kOutStride;
    f.n = (int)n;
    f.K = K;
    f.L = r0->L;
    f.M = r0->M;
    f.u = out_u.as<double>();
    f.coef = out_coef.as<double>();
    f.se = out_se.as<double>();
    f.status = out_status.as<int32_t>();
    f.stats = w.stats;
    if (e == cudaSuccess) e = grt::launch_finalize(fp64, f, stream);
    ++launches;
    if (e != cudaSuccess) {
      why = std::string("step launch: ") + cudaGetErrorString(e);
      return GRT_EDEVICE;
    }
    g0 = g1;
  }
  const cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    why = std::string("step: ") + cudaGetErrorString(e);
    return GRT_EDEVICE;
  }
  return GRT_OK;
}

void grt_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lock(mu);
  while (!stop) {
    // admission: first come, first admitted, while the resident state fits the budget
    while (!pending.empty()) {
      Request *r = pending.front();
      uint64_t prow = 0, orow = 0;
      if (!part_rows.alloc(r->part_rows, &prow)) break;
      if (!out_rows.alloc((uint64_t)r->n, &orow)) {
        part_rows.release(prow, r->part_rows);
        break;
      }
      r->part_row = prow;
      r->out_row = orow;
      uint64_t slot = prow;
      for (int64_t i = 0; i < r->n; ++i) {
        r->part_slot[i] = (uint32_t)slot;
        slot += point_chunks(r->N[i]);
      }
      r->admitted = true;
      pending.pop_front();
      active.push_back(r);
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
    lock.unlock();
    std::string why;
    const int rc = run_step(units, why);
    lock.lock();
    ++steps;
    if (rc != GRT_OK) {
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
      continue;
    }
    // bookkeeping; finished requests take their results off the device and free their rows
    for (const Unit &u : units) {
      Request *r = u.r;
      r->done[u.i] += u.cnt;
      r->remaining -= u.cnt;
      trees_walked += u.cnt;
      if (r->done[u.i] == r->N[u.i]) {
        r->complete[u.i] = 1;
        --r->points_left;
      }
    }
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
      cudaError_t e = cudaMemcpy(r->u.data(), out_u.as<double>() + r->out_row, n * 8, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(r->status.data(), out_status.as<int32_t>() + r->out_row, n * 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy2D(r->coef.data(), K1 * 8, out_coef.as<double>() + r->out_row * kOutStride, kOutStride * 8, K1 * 8,
                         n, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy2D(r->se.data(), K1 * 8, out_se.as<double>() + r->out_row * kOutStride, kOutStride * 8, K1 * 8, n,
                         cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        r->error = GRT_EDEVICE;
        r->error_text = cudaGetErrorString(e);
      }
      part_rows.release(r->part_row, r->part_rows);
      out_rows.release(r->out_row, (uint64_t)r->n);
      r->finished = true;
      r->t_finish = Clock::now();
      active.erase(active.begin() + (ptrdiff_t)k);
    }
    cv_done.notify_all();
  }
}

extern "C" {

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
  s->meta_points = (size_t)std::min<uint64_t>(1ull << 20, std::max<uint64_t>(4096, step_trees / 256));
  const size_t step_bytes = (size_t)step_trees * 9 + 64 * 1024 + s->meta_points * (9 * 4 + 8 + 4 * 8 + 4);
  if (mem_budget_bytes < step_bytes + (1ull << 20)) {
    delete s;
    return GRT_EINVAL;  // the budget must hold the step buffers and some resident state
  }
  const uint64_t resident = mem_budget_bytes - step_bytes;
  const uint64_t part_cap = (resident * 3 / 4) / (kPartStride * 8);
  const uint64_t out_cap = (resident / 4) / ((2 * kOutStride + 2) * 8);
  cudaError_t e;
  if ((e = cudaSetDevice(device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = s->part_pool.ensure(part_cap * kPartStride * 8)) != cudaSuccess ||
      (e = s->out_u.ensure(out_cap * 8)) != cudaSuccess || (e = s->out_status.ensure(out_cap * 4)) != cudaSuccess ||
      (e = s->out_coef.ensure(out_cap * kOutStride * 8)) != cudaSuccess ||
      (e = s->out_se.ensure(out_cap * kOutStride * 8)) != cudaSuccess ||
      (e = s->rec_w.ensure((size_t)step_trees * 8 + 4 * 8 * s->meta_points + 64)) != cudaSuccess ||
      (e = s->rec_o.ensure((size_t)step_trees + 4 * s->meta_points + 64)) != cudaSuccess ||
      (e = s->meta.ensure(9 * (s->meta_points + 1) * 4 + (s->meta_points + 1) * 8)) != cudaSuccess ||
      (e = s->xbuf.ensure(s->meta_points * (GRT_MAX_DIM + 1) * 8)) != cudaSuccess ||
      (e = s->work.ensure(64 + s->meta_points * 4)) != cudaSuccess) {
    s->part_pool.release();
    s->out_u.release();
    s->out_status.release();
    s->out_coef.release();
    s->out_se.release();
    s->rec_w.release();
    s->rec_o.release();
    s->meta.release();
    s->xbuf.release();
    s->work.release();
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return e == cudaErrorMemoryAllocation ? GRT_ENOMEM : GRT_EDEVICE;
  }
  s->part_rows.init(part_cap);
  s->out_rows.init(out_cap);
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
  s->part_pool.release();
  s->out_u.release();
  s->out_status.release();
  s->out_coef.release();
  s->out_se.release();
  s->rec_w.release();
  s->rec_o.release();
  s->meta.release();
  s->xbuf.release();
  s->work.release();
  if (s->stream) cudaStreamDestroy(s->stream);
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
  r->part_slot.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (ntrees[i] > GRT_MAX_TREES_PER_POINT || !std::isfinite(t[i]) || t[i] < 0.0) {
      delete r;
      return s->set_error(GRT_EINVAL, "ntrees[i] <= 2^31 - 1 and finite t[i] >= 0 required");
    }
    r->N[i] = (uint32_t)ntrees[i];
    r->remaining += ntrees[i];
    r->part_rows += point_chunks(r->N[i]);
  }
  r->points_left = n;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fatal) {
      delete r;
      return s->set_error(s->fatal, "server stopped after a device error: " + s->err);
    }
    if (r->part_rows > s->part_rows.capacity() || (uint64_t)n > s->out_rows.capacity()) {
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

int grt_poll(grt_server *s, uint64_t request_id, int timeout_ms, double *u_out, double *coef_out, double *se_out,
             int32_t *status_out, double *latency_s) {
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
  if (rc == GRT_OK) {
    const size_t n = (size_t)r->n, K1 = (size_t)r->K + 1;
    if (u_out && n) std::memcpy(u_out, r->u.data(), n * 8);
    if (status_out && n) std::memcpy(status_out, r->status.data(), n * 4);
    if (coef_out && n) std::memcpy(coef_out, r->coef.data(), n * K1 * 8);
    if (se_out && n) std::memcpy(se_out, r->se.data(), n * K1 * 8);
  } else {
    s->err = r->error_text;
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_finish - r->t_submit).count();
  s->reqs.erase(it);
  delete r;
  return rc;
}

int grt_server_stats(grt_server *s, uint64_t *steps, uint64_t *trees, uint64_t *launches, uint64_t *resident_bytes,
                     uint64_t *pending_requests, uint64_t *active_requests) {
  if (!s) return GRT_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (steps) *steps = s->steps;
  if (trees) *trees = s->trees_walked;
  if (launches) *launches = s->launches;
  if (resident_bytes)
    *resident_bytes = s->part_rows.used() * kPartStride * 8 + s->out_rows.used() * (2 * kOutStride + 2) * 8;
  if (pending_requests) *pending_requests = s->pending.size();
  if (active_requests) *active_requests = s->active.size();
  return GRT_OK;
}

}  // extern "C"
