// mm_server.cu -- the serving form: a request loop over one day's events kept
// resident on the device. Each request asks for the covariance / correlation
// (Algorithm 3) of an asset subset over a time window at a cutoff N (given,
// from Eq. (19) for a sampling interval, or the window's Nyquist cutoff of
// Algorithm 2). Times are rescaled with the request's window (t0, t1), so an
// asset's coefficients do not depend on which other assets are requested.
//
// Continuous batching: a native scheduler thread admits queued requests into
// execution slots as slots free up, and every slot runs its request on its own
// CUDA stream, so the work of requests that arrived at different times
// overlaps on the GPU. The number of slots comes from the HBM budget: each
// slot holds the workspace of the largest admissible request (asset count,
// events in the window, cutoff), and a request enters only a free slot.
// Requests complete out of order; the caller polls completions with their
// submit / start / finish times (host clock), from which p50 / p99 latency
// follow.
//
// Resident coefficients: with a cache, each requested asset's coefficients
// over the request's window at its cutoff are kept in a device row keyed by
// (asset, t0, t1, N); a request computes only the assets it does not find,
// writes them into fresh rows, and gathers all its rows for the contraction.
// New rows become visible to other requests when their request has finished
// (so no slot reads a row another slot is still writing); rows in use are
// pinned; unpinned rows are evicted least recently used first. The index is
// touched only by the scheduler thread.
#include <atomic>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "mm_common.cuh"
#include "server_cache.h"

using namespace mmgpu;

namespace {

// Window of each requested asset in the resident store (lo = first event
// with t >= t0, count = events with t <= t1 from there), prefix-summed into
// the request's CSR offsets. One block; an invalid asset id or more events
// than the slot holds empties the request and flags bad input.
__global__ void k_window_offsets(const int64_t* __restrict__ off_all, const double* __restrict__ t_all, int D_all,
                                 const int32_t* __restrict__ assets, int n, double t0, double t1, int64_t cap,
                                 int64_t* __restrict__ lo_out, int64_t* __restrict__ off_req, int* status) {
  extern __shared__ int64_t s_cnt[];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int a = assets[i];
    int64_t lo = 0, cnt = 0;
    if (a < 0 || a >= D_all) {
      atomicOr(&s_bad, 1);
    } else {
      const int64_t b0 = off_all[a], b1 = off_all[a + 1];
      int64_t l = b0, h = b1;  // first t >= t0
      while (l < h) {
        const int64_t m = (l + h) >> 1;
        if (t_all[m] < t0) l = m + 1;
        else h = m;
      }
      lo = l;
      h = b1;  // first t > t1
      while (l < h) {
        const int64_t m = (l + h) >> 1;
        if (t_all[m] <= t1) l = m + 1;
        else h = m;
      }
      cnt = l - lo;
    }
    lo_out[i] = lo;
    s_cnt[i] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    off_req[0] = 0;
    for (int i = 0; i < n; ++i) {
      acc += s_cnt[i];
      off_req[i + 1] = acc;
    }
    if (acc > cap) s_bad = 1;
    if (s_bad) {
      for (int i = 0; i <= n; ++i) off_req[i] = 0;
      atomicOr(status, ST_BAD_OFFSETS);
    }
  }
}

// Copy each requested asset's window of events (block i: asset i).
__global__ void k_window_copy(const int64_t* __restrict__ lo, const int64_t* __restrict__ off_req,
                              const double* __restrict__ t_all, const double* __restrict__ p_all,
                              double* __restrict__ t_req, double* __restrict__ p_req) {
  const int i = blockIdx.x;
  const int64_t src = lo[i], dst = off_req[i], cnt = off_req[i + 1] - off_req[i];
  for (int64_t h = threadIdx.x; h < cnt; h += blockDim.x) {
    t_req[dst + h] = t_all[src + h];
    p_req[dst + h] = p_all[src + h];
  }
}

// Coefficient rows between a dense [n][ld] matrix and the cache's rows
// (8-byte units: complex64 or complex128 coefficients). Block i: row i.
__global__ void k_rows_to_cache(const unsigned long long* __restrict__ src, int64_t src_ld,
                                unsigned long long* __restrict__ cache, int64_t cache_ld,
                                const int32_t* __restrict__ rows, int64_t width) {
  const int i = blockIdx.x;
  const unsigned long long* a = src + (int64_t)i * src_ld;
  unsigned long long* b = cache + (int64_t)rows[i] * cache_ld;
  for (int64_t j = threadIdx.x; j < width; j += blockDim.x) b[j] = a[j];
}

__global__ void k_rows_from_cache(const unsigned long long* __restrict__ cache, int64_t cache_ld,
                                  const int32_t* __restrict__ rows, unsigned long long* __restrict__ dst,
                                  int64_t dst_ld, int64_t width) {
  const int i = blockIdx.x;
  const unsigned long long* a = cache + (int64_t)rows[i] * cache_ld;
  unsigned long long* b = dst + (int64_t)i * dst_ld;
  for (int64_t j = threadIdx.x; j < width; j += blockDim.x) b[j] = a[j];
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  int64_t ticket = 0;
  double t0 = 0, t1 = 0, dt = 0;
  int N = 0;
  std::vector<int32_t> assets;
  void* h_R = nullptr;
  void* h_S = nullptr;
  double t_submit = 0, t_start = 0;
};

struct Slot {
  mm_plan p = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  int32_t* d_assets = nullptr;
  int64_t* d_lo = nullptr;
  int64_t* d_off = nullptr;
  double* d_t = nullptr;
  double* d_p = nullptr;
  void* d_coef = nullptr;
  void* d_S = nullptr;
  void* d_R = nullptr;
  int32_t* h_assets = nullptr;  // pinned
  void* h_S = nullptr;          // pinned
  void* h_R = nullptr;          // pinned
  int* h_status = nullptr;      // pinned
  int32_t* d_rows = nullptr;    // cache rows of the request's computed assets, then of all its assets
  int32_t* h_rows = nullptr;    // pinned staging of d_rows
  std::vector<int> pinned;      // cache rows this request reads (found in the index)
  std::vector<int> reserved;    // cache rows this request writes (published when it finishes)
  bool busy = false;
  mm_status early = MM_OK;      // error found while enqueueing
  int N_used = 0;
  Req req;
};

}  // namespace

struct mm_server_s {
  mm_server_desc desc{};
  int dev = 0;
  size_t rs = 4;
  int64_t req_events = 0;  // events a slot holds
  int64_t* d_off_all = nullptr;
  double* d_t_all = nullptr;
  double* d_p_all = nullptr;
  bool loaded = false;
  std::vector<Slot> slots;
  int64_t slot_bytes = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> queue;
  std::deque<mm_completion> done;
  std::thread th;
  bool stop = false;
  int64_t next_ticket = 1;
  int64_t submitted = 0, completed = 0;
  std::atomic<int64_t> launches{0};  // kernels launched for requests (start() runs outside mu)
  int inflight = 0, peak_inflight = 0;
  double t_origin = 0;
  // resident coefficients (the index is used by the scheduler thread only,
  // or under mu while idle)
  void* d_cache = nullptr;  // cache_rows x (N_max + 1) coefficients
  CoefCache cache;
  std::atomic<int64_t> cache_hits{0}, cache_misses{0};
};

namespace {

// A finished request's rows: the ones it read are unpinned; the ones it
// wrote are published (unless the request failed, or the same key was
// published meanwhile) or returned.
void cache_release(mm_server s, Slot& sl, bool ok) {
  for (int r : sl.pinned) s->cache.unpin(r);
  for (int r : sl.reserved) s->cache.finish_reserved(r, ok);
  sl.pinned.clear();
  sl.reserved.clear();
}

void free_slot(Slot& s) {
  if (s.p) mm_destroy(s.p);
  void* dptrs[] = {s.d_assets, s.d_lo, s.d_off, s.d_t, s.d_p, s.d_coef, s.d_S, s.d_R, s.d_rows};
  for (void* q : dptrs)
    if (q) cudaFree(q);
  void* hptrs[] = {s.h_assets, s.h_S, s.h_R, s.h_status, s.h_rows};
  for (void* q : hptrs)
    if (q) cudaFreeHost(q);
  if (s.done) cudaEventDestroy(s.done);
  if (s.st) cudaStreamDestroy(s.st);
  s = Slot{};
}

mm_status make_slot(mm_server s, Slot& sl, int64_t* bytes) {
  const mm_server_desc& d = s->desc;
  mm_plan_desc pd{};
  pd.D = d.D;
  pd.N_max = d.N_max;
  pd.max_events = s->req_events;
  pd.tol = d.tol;
  pd.kernel = d.kernel;
  pd.basis = d.basis;
  pd.prec = d.prec;
  mm_status r = plan_create_no_staging(&pd, &sl.p);
  if (r != MM_OK) return r;
  mm_plan_info info;
  mm_plan_get_info(sl.p, &info);
  const size_t D = (size_t)d.D, E = (size_t)std::max<int64_t>(s->req_events, 1);
  const size_t cs = 2 * s->rs;
  int64_t b = info.workspace_bytes;
  auto A = [&](void** ptr, size_t n) -> bool {
    if (cudaMalloc(ptr, n) != cudaSuccess) return false;
    b += (int64_t)n;
    return true;
  };
  bool ok = A((void**)&sl.d_assets, D * 4) && A((void**)&sl.d_lo, D * 8) && A((void**)&sl.d_off, (D + 1) * 8) &&
            A((void**)&sl.d_t, E * 8) && A((void**)&sl.d_p, E * 8) &&
            A(&sl.d_coef, D * ((size_t)d.N_max + 1) * cs) && A(&sl.d_S, D * D * s->rs) && A(&sl.d_R, D * D * s->rs) &&
            A((void**)&sl.d_rows, 2 * D * 4);
  ok = ok && cudaMallocHost((void**)&sl.h_rows, 2 * D * 4) == cudaSuccess &&
       cudaMallocHost((void**)&sl.h_assets, D * 4) == cudaSuccess &&
       cudaMallocHost(&sl.h_S, D * D * s->rs) == cudaSuccess && cudaMallocHost(&sl.h_R, D * D * s->rs) == cudaSuccess &&
       cudaMallocHost((void**)&sl.h_status, 16) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return MM_ERR_OOM;
  }
  *bytes = b;
  return MM_OK;
}

// Enqueue one request on its slot's stream (called by the scheduler thread
// without the server lock). Errors found on the host end the request at once.
void start(mm_server s, Slot& sl, Req&& rq) {
  sl.req = std::move(rq);
  sl.req.t_start = now_s() - s->t_origin;
  sl.busy = true;
  sl.early = MM_OK;
  sl.N_used = 0;
  sl.pinned.clear();
  sl.reserved.clear();
  const int n = (int)sl.req.assets.size();
  cudaStream_t st = sl.st;
  auto fail = [&](mm_status r) {
    sl.early = r;
    cudaEventRecord(sl.done, st);
  };
  int N = sl.req.N;
  if (N <= 0 && sl.req.dt > 0.0) {
    // Eq. (19) for the sampling interval dt over the window length
    N = (int)floor(0.5 * ((sl.req.t1 - sl.req.t0) / sl.req.dt - 1.0));
    if (N < 1) N = 1;
  }
  if (N > s->desc.N_max) N = s->desc.N_max;

  // resident coefficients: with the cutoff known on the host, the assets
  // found in the cache are read from their rows and only the others are
  // computed (into rows reserved for them)
  bool cached = s->cache.size() > 0 && N > 0;
  std::vector<int> compute;  // positions in the request of the assets computed here
  std::vector<int> row_of;
  if (cached) {
    row_of.assign(n, -1);
    for (int i = 0; i < n; ++i) {
      CacheKey k;
      k.asset = sl.req.assets[i];
      k.N = N;
      k.t0 = sl.req.t0;
      k.t1 = sl.req.t1;
      const int r = s->cache.acquire(k);
      if (r >= 0) {
        sl.pinned.push_back(r);
        row_of[i] = r;
      } else {
        compute.push_back(i);
      }
    }
    for (int i : compute) {
      CacheKey k;
      k.asset = sl.req.assets[i];
      k.N = N;
      k.t0 = sl.req.t0;
      k.t1 = sl.req.t1;
      const int r = s->cache.reserve(k);
      if (r < 0) {  // every row in use: serve this request without the cache
        cache_release(s, sl, false);
        cached = false;
        break;
      }
      sl.reserved.push_back(r);
      row_of[i] = r;
    }
  }
  if (!cached) {
    compute.resize(n);
    for (int i = 0; i < n; ++i) compute[i] = i;
  }
  const int nc = (int)compute.size();
  for (int j = 0; j < nc; ++j) sl.h_assets[j] = sl.req.assets[compute[j]];

  mm_plan_info pi0{};
  mm_plan_get_info(sl.p, &pi0);
  int* status = plan_status_word(sl.p);
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return fail(MM_ERR_CUDA);
  int32_t Nu = N;
  mm_status r = MM_OK;
  if (nc > 0) {
    if (cudaMemcpyAsync(sl.d_assets, sl.h_assets, (size_t)nc * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(MM_ERR_CUDA);
    k_window_offsets<<<1, 512, (size_t)nc * 8, st>>>(s->d_off_all, s->d_t_all, s->desc.D, sl.d_assets, nc,
                                                     sl.req.t0, sl.req.t1, s->req_events, sl.d_lo, sl.d_off, status);
    k_window_copy<<<nc, 256, 0, st>>>(sl.d_lo, sl.d_off, s->d_t_all, s->d_p_all, sl.d_t, sl.d_p);
    if (cudaGetLastError() != cudaSuccess) return fail(MM_ERR_CUDA);
    s->launches.fetch_add(2);
    r = plan_set_active_assets(sl.p, nc);
    if (r != MM_OK) return fail(r);
    r = mm_coeffs(sl.p, sl.d_off, sl.d_t, sl.d_p, N, sl.req.t0, sl.req.t1, sl.d_coef, &Nu, st);
    if (r == MM_ERR_CUTOFF && N <= 0) {
      // a window Nyquist cutoff above N_max: serve it at N_max
      r = mm_coeffs(sl.p, sl.d_off, sl.d_t, sl.d_p, s->desc.N_max, sl.req.t0, sl.req.t1, sl.d_coef, &Nu, st);
    }
    if (r != MM_OK) return fail(r);
  }
  if (cached) {
    // computed rows into their cache rows, then every requested row (in
    // request order) into the contraction's operand
    const int D = s->desc.D;
    for (int j = 0; j < nc; ++j) sl.h_rows[j] = row_of[compute[j]];
    for (int i = 0; i < n; ++i) sl.h_rows[D + i] = row_of[i];
    const int64_t u = (int64_t)(2 * s->rs) / 8;  // 8-byte units per coefficient
    const int64_t width = (int64_t)(N + 1) * u, cld = (int64_t)(s->desc.N_max + 1) * u;
    if (cudaMemcpyAsync(sl.d_rows, sl.h_rows, (size_t)2 * D * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(MM_ERR_CUDA);
    if (nc > 0)
      k_rows_to_cache<<<nc, 256, 0, st>>>((const unsigned long long*)sl.d_coef, width,
                                          (unsigned long long*)s->d_cache, cld, sl.d_rows, width);
    k_rows_from_cache<<<n, 256, 0, st>>>((const unsigned long long*)s->d_cache, cld, sl.d_rows + D,
                                         (unsigned long long*)sl.d_coef, width, width);
    if (cudaGetLastError() != cudaSuccess) return fail(MM_ERR_CUDA);
    s->launches.fetch_add(nc > 0 ? 2 : 1);
    s->cache_hits.fetch_add(n - nc);
    s->cache_misses.fetch_add(nc);
    r = plan_set_active_assets(sl.p, n);
    if (r != MM_OK) return fail(r);
  }
  sl.N_used = Nu;
  r = mm_corr(sl.p, sl.d_coef, Nu, sl.req.h_S ? sl.d_S : nullptr, sl.d_R, st);
  if (r != MM_OK) return fail(r);
  mm_plan_info pi1{};
  if (mm_plan_get_info(sl.p, &pi1) == MM_OK) s->launches.fetch_add(pi1.launches - pi0.launches);
  const size_t bytes = (size_t)n * n * s->rs;
  if (cudaMemcpyAsync(sl.h_R, sl.d_R, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (sl.req.h_S && cudaMemcpyAsync(sl.h_S, sl.d_S, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      cudaMemcpyAsync(sl.h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaEventRecord(sl.done, st) != cudaSuccess)
    return fail(MM_ERR_CUDA);
}

// A finished slot: results to the caller's buffers, a completion record.
mm_completion finish(mm_server s, Slot& sl) {
  mm_completion c{};
  c.ticket = sl.req.ticket;
  c.n_assets = (int32_t)sl.req.assets.size();
  c.N = sl.N_used;
  c.t_submit = sl.req.t_submit;
  c.t_start = sl.req.t_start;
  c.t_done = now_s() - s->t_origin;
  if (sl.early != MM_OK) {
    c.status = sl.early;
  } else {
    c.status = plan_flags_to_status(*sl.h_status);
    const size_t bytes = (size_t)c.n_assets * c.n_assets * s->rs;
    if (sl.req.h_R) memcpy(sl.req.h_R, sl.h_R, bytes);
    if (sl.req.h_S) memcpy(sl.req.h_S, sl.h_S, bytes);
  }
  // zero variance concerns R only: the request's coefficients are valid
  cache_release(s, sl, c.status == MM_OK || c.status == MM_ERR_ZERO_VARIANCE);
  sl.busy = false;
  return c;
}

void scheduler(mm_server s) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progress = false;
    for (Slot& sl : s->slots) {
      if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) {
        mm_completion c = finish(s, sl);
        s->done.push_back(c);
        s->completed += 1;
        s->inflight -= 1;
        progress = true;
      }
    }
    if (progress) s->cv.notify_all();
    for (Slot& sl : s->slots) {
      if (s->queue.empty()) break;
      if (sl.busy) continue;
      Req rq = std::move(s->queue.front());
      s->queue.pop_front();
      s->inflight += 1;
      s->peak_inflight = std::max(s->peak_inflight, s->inflight);
      sl.busy = true;
      lk.unlock();
      start(s, sl, std::move(rq));
      lk.lock();
      progress = true;
    }
    if (s->stop && s->queue.empty() && s->inflight == 0) break;
    if (!progress) {
      if (s->inflight > 0) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(5));
        lk.lock();
      } else {
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
      }
    }
  }
}

}  // namespace

extern "C" {

mm_status mm_server_create(const mm_server_desc* desc, mm_server* out) {
  if (!out) return MM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return MM_ERR_INVALID_ARG;
  const mm_server_desc& d = *desc;
  if (d.D < 1 || d.D > 4096 || d.N_max < 1 || d.max_events < 1 || d.request_max_events < 0 ||
      d.hbm_budget < 0 || d.max_slots < 1 || d.max_slots > 64 || d.cache_rows < 0 || d.cache_rows > (1 << 22))
    return MM_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (d.reserved[i] != 0) return MM_ERR_INVALID_ARG;
  if (d.prec < MM_PREC_FP64 || d.prec > MM_PREC_MIXED_3XTF32) return MM_ERR_INVALID_ARG;
  mm_server s = new mm_server_s();
  s->desc = d;
  s->rs = d.prec == MM_PREC_FP64 ? 8 : 4;
  s->req_events = d.request_max_events > 0 ? std::min(d.request_max_events, d.max_events) : d.max_events;
  s->t_origin = now_s();
  if (cudaGetDevice(&s->dev) != cudaSuccess || cudaMalloc((void**)&s->d_off_all, ((size_t)d.D + 1) * 8) != cudaSuccess ||
      cudaMalloc((void**)&s->d_t_all, (size_t)d.max_events * 8) != cudaSuccess ||
      cudaMalloc((void**)&s->d_p_all, (size_t)d.max_events * 8) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->d_off_all);
    cudaFree(s->d_t_all);
    delete s;
    return MM_ERR_OOM;
  }
  if (d.cache_rows > 0) {
    const size_t cs = 2 * s->rs;
    if (cudaMalloc(&s->d_cache, (size_t)d.cache_rows * ((size_t)d.N_max + 1) * cs) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(s->d_off_all);
      cudaFree(s->d_t_all);
      cudaFree(s->d_p_all);
      delete s;
      return MM_ERR_OOM;
    }
    s->cache.reset(d.cache_rows);
  }
  // slots: as many as the budget holds (at least one), each sized for the
  // largest admissible request
  mm_status r = MM_OK;
  for (int i = 0; i < d.max_slots; ++i) {
    Slot sl;
    int64_t b = 0;
    r = make_slot(s, sl, &b);
    if (r != MM_OK) {
      free_slot(sl);
      break;
    }
    s->slot_bytes = b;
    s->slots.push_back(sl);
    if (d.hbm_budget > 0 && (int64_t)(s->slots.size() + 1) * b > d.hbm_budget) break;
  }
  if (s->slots.empty()) {
    cudaFree(s->d_off_all);
    cudaFree(s->d_t_all);
    cudaFree(s->d_p_all);
    cudaFree(s->d_cache);
    delete s;
    return r != MM_OK ? r : MM_ERR_OOM;
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return MM_OK;
}

mm_status mm_server_load(mm_server s, const int64_t* h_offsets, const double* h_t, const double* h_logp) {
  if (!s || !h_offsets || !h_t || !h_logp) return MM_ERR_INVALID_ARG;
  const int D = s->desc.D;
  if (h_offsets[0] != 0 || h_offsets[D] > s->desc.max_events) return MM_ERR_INVALID_ARG;
  for (int i = 0; i < D; ++i) {
    if (h_offsets[i + 1] < h_offsets[i]) return MM_ERR_INVALID_ARG;
    for (int64_t h = h_offsets[i]; h + 1 < h_offsets[i + 1]; ++h)
      if (!(h_t[h] < h_t[h + 1])) return h_t[h] == h_t[h + 1] ? MM_ERR_DUPLICATE_TIME : MM_ERR_UNSORTED;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->inflight > 0 || !s->queue.empty()) return MM_ERR_INVALID_ARG;  // reload only while idle
  const size_t E = (size_t)h_offsets[D];
  if (cudaMemcpy(s->d_off_all, h_offsets, ((size_t)D + 1) * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_t_all, h_t, E * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_p_all, h_logp, E * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    return MM_ERR_CUDA;
  s->cache.clear();  // the rows were of the previous store
  s->loaded = true;
  return MM_OK;
}

mm_status mm_server_submit(mm_server s, const mm_request* rq, int64_t* ticket) {
  if (!s || !rq || !ticket) return MM_ERR_INVALID_ARG;
  if (!s->loaded) return MM_ERR_INVALID_ARG;
  if (!(rq->t1 > rq->t0) || !isfinite(rq->t0) || !isfinite(rq->t1)) return MM_ERR_INVALID_ARG;
  if (rq->n_assets < 1 || rq->n_assets > s->desc.D || !rq->assets || !rq->h_R) return MM_ERR_INVALID_ARG;
  if (rq->N < 0 || rq->N > s->desc.N_max || !(rq->dt_equiv >= 0.0)) return MM_ERR_INVALID_ARG;
  Req r;
  r.t0 = rq->t0;
  r.t1 = rq->t1;
  r.dt = rq->dt_equiv;
  r.N = rq->N;
  r.assets.assign(rq->assets, rq->assets + rq->n_assets);
  r.h_R = rq->h_R;
  r.h_S = rq->h_sigma_or_null;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r.ticket = s->next_ticket++;
    r.t_submit = now_s() - s->t_origin;
    *ticket = r.ticket;
    s->queue.push_back(std::move(r));
    s->submitted += 1;
  }
  s->cv.notify_all();
  return MM_OK;
}

mm_status mm_server_poll(mm_server s, mm_completion* out, int32_t max, int32_t* n_out, double wait_s) {
  if (!s || !out || !n_out || max < 1) return MM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_s > 0.0)
    s->cv.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !s->done.empty(); });
  int n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  *n_out = n;
  return MM_OK;
}

mm_status mm_server_get_stats(mm_server s, mm_server_stats* st) {
  if (!s || !st) return MM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof(*st));
  st->slots = (int32_t)s->slots.size();
  st->inflight = s->inflight;
  st->peak_inflight = s->peak_inflight;
  st->queued = (int32_t)s->queue.size();
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->slot_bytes = s->slot_bytes;
  st->resident_bytes = (int64_t)(s->desc.D + 1) * 8 + 16 * s->desc.max_events;
  st->launches = s->launches.load();
  st->cache_hits = s->cache_hits.load();
  st->cache_misses = s->cache_misses.load();
  return MM_OK;
}

mm_status mm_server_destroy(mm_server s) {
  if (!s) return MM_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->dev);
  for (Slot& sl : s->slots) free_slot(sl);
  cudaFree(s->d_off_all);
  cudaFree(s->d_t_all);
  cudaFree(s->d_p_all);
  cudaFree(s->d_cache);
  delete s;
  return MM_OK;
}

}  // extern "C"
