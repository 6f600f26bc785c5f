// Request-serving engine on top of the C ABI (os3d_forward / os3d_inverse).
//
// A worker thread takes requests (a host volume, its grid and orientation
// set) in arrival order and admits each one as soon as a stream slot and
// enough of the device arena are free; admitted requests run concurrently,
// one per stream: host-to-device copy of the volume, forward transform into a
// score held in the arena, exact inverse, device-to-host copy of the
// reconstruction. Completion is signalled by a host function enqueued behind
// the copy. Wavelet banks are cached per (grid, orientation set), up to a
// byte budget (least recently used idle banks are destroyed beyond it); the
// arena is allocated once at creation, so requests allocate no device memory.
// Placement: every bank keeps a short list of "home" offsets in the arena, the
// places its earlier requests occupied; a request goes to the first free home
// of its bank, else first fit (which becomes a new home while the list has
// room). With use_graphs, the kernel sequence of forward + inverse of a (bank,
// home) is captured into a CUDA graph on its first use and replayed by every
// later request placed there: one launch instead of about fifty.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>
#include "../../include/os3d.h"
#include "os3d_kernels.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// first-fit allocator over [0, size) with coalescing
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  // [off, off + n) exactly, if it lies inside one free range
  bool alloc_at(size_t off, size_t n) {
    auto it = free_.upper_bound(off);
    if (it == free_.begin()) return false;
    --it;
    const size_t s = it->first, len = it->second;
    if (off < s || off + n > s + len) return false;
    free_.erase(it);
    if (off > s) free_[s] = off - s;
    if (s + len > off + n) free_[off + n] = s + len - (off + n);
    return true;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

struct BankEntry;

struct Request {
  long long id = 0;
  int dims[3] = {0, 0, 0};
  int subdiv = 0;
  const float* f = nullptr;
  float* f_out = nullptr;
  Clock::time_point t_submit, t_done;
  size_t off = 0, bytes = 0;
  int slot = -1;
  BankEntry* bank = nullptr;   // set at admission; its in-flight count covers the request
  bool done = false;
  os3d_status status = OS3D_OK;
};

struct BankEntry {
  os3d_bank* bank = nullptr;
  int n_o = 0;
  size_t ws_bytes = 0, footprint = 0, resident = 0;
  int inflight = 0;                  // admitted requests not yet retired (worker thread)
  unsigned long long last_use = 0;   // admission counter value of the latest use
  std::vector<size_t> homes;         // arena offsets whose graphs belong to this bank
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;   // kernel launches the graph replays
};
constexpr size_t kMaxGraphs = 512;

}  // namespace

struct os3d_server {
  os3d_server_config cfg{};
  os3d_params params{};
  int dev = 0;
  void* arena_base = nullptr;
  std::unique_ptr<Arena> arena;
  std::vector<cudaStream_t> streams;
  std::vector<std::shared_ptr<Request>> slot_req;   // in-flight request per stream slot
  cudaStream_t bank_stream = nullptr;
  std::map<std::tuple<int, int, int, int>, BankEntry> banks;
  size_t bank_bytes = 0;                 // resident device bytes of the cached banks
  unsigned long long admissions = 0;
  std::map<std::pair<const os3d_bank*, size_t>, GraphEntry> graphs;   // worker thread only
  long long n_done = 0, n_captured = 0, n_replayed = 0;                // under mu
  std::deque<std::shared_ptr<Request>> pending;
  std::map<long long, std::shared_ptr<Request>> all;
  std::mutex mu;
  std::condition_variable cv;        // worker wake-ups
  std::condition_variable done_cv;   // waiters
  bool stop = false;
  long long next_id = 1;
  std::thread worker;

  // completed by a host function on the request's stream
  struct Done {
    os3d_server* s;
    Request* r;
  };
  static void CUDART_CB on_done(void* p) {
    std::unique_ptr<Done> d(static_cast<Done*>(p));
    std::lock_guard<std::mutex> lk(d->s->mu);
    d->r->t_done = Clock::now();
    d->r->done = true;
    d->s->n_done += 1;
    d->s->cv.notify_all();
    d->s->done_cv.notify_all();
  }

  // destroys idle cached banks, least recently used first, until the cache
  // plus `extra` bytes fits the budget. Worker thread, with mu NOT held:
  // destroying a bank frees device memory, which may wait for the host
  // functions of in-flight requests, and those take mu. Banks, their
  // in-flight counts and the graphs are touched by the worker thread only.
  void evict_banks(size_t extra, const BankEntry* keep) {
    while (bank_bytes + extra > cfg.bank_cache_bytes) {
      auto victim = banks.end();
      for (auto it = banks.begin(); it != banks.end(); ++it)
        if (it->second.inflight == 0 && &it->second != keep &&
            (victim == banks.end() || it->second.last_use < victim->second.last_use))
          victim = it;
      if (victim == banks.end()) return;   // the rest is in use
      for (auto g = graphs.begin(); g != graphs.end();) {
        if (g->first.first == victim->second.bank) {
          cudaGraphExecDestroy(g->second.exec);
          g = graphs.erase(g);
        } else {
          ++g;
        }
      }
      os3d_destroy_bank(victim->second.bank);
      bank_bytes -= victim->second.resident;
      banks.erase(victim);
    }
  }

  // the bank of (grid, orientation set), made on first use (worker thread only)
  os3d_status bank_for(const Request& r, BankEntry** out) {
    const auto key = std::make_tuple(r.dims[0], r.dims[1], r.dims[2], r.subdiv);
    auto it = banks.find(key);
    if (it == banks.end()) {
      int n_o = 0;
      os3d_icosa_orientations(r.subdiv, nullptr, 0, &n_o);
      std::vector<double> V(3 * (size_t)std::max(n_o, 1));
      os3d_status st = os3d_icosa_orientations(r.subdiv, V.data(), n_o, &n_o);
      if (st != OS3D_OK) return st;
      BankEntry e;
      st = os3d_make_wavelets(r.dims, V.data(), n_o, &params, bank_stream, &e.bank);
      if (st != OS3D_OK) return st;
      e.n_o = n_o;
      os3d_bank_info(e.bank, &e.ws_bytes, nullptr);
      os3d_bank_resident_bytes(e.bank, &e.resident);
      const size_t nvox = (size_t)r.dims[0] * r.dims[1] * r.dims[2];
      const size_t esz = cfg.udtype == OS3D_U_BF16X2 ? 4 : 8;
      e.footprint = align_up((size_t)e.n_o * nvox * esz) + 2 * align_up(nvox * sizeof(float)) +
                    align_up(e.ws_bytes);
      evict_banks(e.resident, nullptr);
      bank_bytes += e.resident;
      it = banks.emplace(key, e).first;
    }
    *out = &it->second;
    return OS3D_OK;
  }

  // enqueue the whole request on stream slot k (worker thread, lock not held)
  os3d_status launch(Request& r, const BankEntry& e, int k) {
    cudaStream_t s = streams[k];
    const size_t nvox = (size_t)r.dims[0] * r.dims[1] * r.dims[2];
    const size_t esz = cfg.udtype == OS3D_U_BF16X2 ? 4 : 8;
    char* base = static_cast<char*>(arena_base) + r.off;
    void* U = base;
    float* fin = reinterpret_cast<float*>(base + align_up((size_t)e.n_o * nvox * esz));
    float* fout = fin + align_up(nvox * sizeof(float)) / sizeof(float);
    void* ws = reinterpret_cast<char*>(fout) + align_up(nvox * sizeof(float));
    if (cudaMemcpyAsync(fin, r.f, nvox * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return OS3D_ECUDA;
    auto transforms = [&]() {
      os3d_status st = os3d_forward(e.bank, fin, 1, U, (os3d_udtype)cfg.udtype, ws, s);
      if (st == OS3D_OK) st = os3d_inverse(e.bank, U, (os3d_udtype)cfg.udtype, 1, fout, ws, s);
      return st;
    };
    const auto key = std::make_pair((const os3d_bank*)e.bank, r.off);
    const bool home = std::find(e.homes.begin(), e.homes.end(), r.off) != e.homes.end();
    const bool use_graph = cfg.use_graphs && home && !os3d::profiling_enabled();
    if (use_graph) {
      auto it = graphs.find(key);
      if (it == graphs.end()) {
        if (graphs.size() >= kMaxGraphs) drop_graphs();
        GraphEntry g;
        const unsigned long long l0 = os3d_launch_count();
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return OS3D_ECUDA;
        const os3d_status st = transforms();
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st != OS3D_OK || ce != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          cudaGetLastError();
          return st != OS3D_OK ? st : OS3D_ECUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return OS3D_ECUDA;
        // the capture counted its kernels once; the first replay executes them
        g.kernels = os3d_launch_count() - l0;
        it = graphs.emplace(key, g).first;
        std::lock_guard<std::mutex> lk(mu);
        n_captured += 1;
      } else {
        os3d::add_launch_count(it->second.kernels);
        std::lock_guard<std::mutex> lk(mu);
        n_replayed += 1;
      }
      if (cudaGraphLaunch(it->second.exec, s) != cudaSuccess) return OS3D_ECUDA;
    } else {
      const os3d_status st = transforms();
      if (st != OS3D_OK) return st;
    }
    if (cudaMemcpyAsync(r.f_out, fout, nvox * sizeof(float), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
      return OS3D_ECUDA;
    if (cudaLaunchHostFunc(s, on_done, new Done{this, &r}) != cudaSuccess) return OS3D_ECUDA;
    return OS3D_OK;
  }

  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }

  void run() {
    cudaSetDevice(dev);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      // retire finished requests: give back their arena space and stream slot
      for (auto& r : slot_req) {
        if (r && r->done) {
          arena->release(r->off, r->bytes);
          if (r->bank) r->bank->inflight -= 1;
          r.reset();
        }
      }
      if (stop && pending.empty()) {
        bool busy = false;
        for (auto& r : slot_req) busy = busy || r;
        if (!busy) break;
      }
      // admit in arrival order while a slot and arena space are free
      bool admitted = false;
      while (!pending.empty()) {
        int k = -1;
        for (int i = 0; i < (int)slot_req.size(); ++i)
          if (!slot_req[i]) {
            k = i;
            break;
          }
        if (k < 0) break;
        std::shared_ptr<Request> r = pending.front();
        BankEntry* e = nullptr;
        lk.unlock();
        os3d_status st = bank_for(*r, &e);
        lk.lock();
        if (st != OS3D_OK) {
          pending.pop_front();
          r->status = st;
          r->done = true;
          r->t_done = Clock::now();
          done_cv.notify_all();
          continue;
        }
        const size_t need = e->footprint;
        size_t off = 0;
        bool placed = false;
        for (size_t h : e->homes)
          if (arena->alloc_at(h, need)) {
            off = h;
            placed = true;
            break;
          }
        if (!placed && need <= cfg.arena_bytes && arena->alloc(need, &off)) {
          placed = true;
          if ((int)e->homes.size() < 2 * cfg.max_inflight) e->homes.push_back(off);
        }
        if (!placed) {
          if (need > cfg.arena_bytes) {   // can never fit
            pending.pop_front();
            r->status = OS3D_ENOMEM;
            r->done = true;
            r->t_done = Clock::now();
            done_cv.notify_all();
            continue;
          }
          break;   // wait for space
        }
        pending.pop_front();
        r->off = off;
        r->bytes = need;
        r->slot = k;
        r->bank = e;
        e->inflight += 1;
        e->last_use = ++admissions;
        slot_req[k] = r;
        lk.unlock();
        st = launch(*r, *e, k);
        lk.lock();
        if (st != OS3D_OK) {
          // the stream may hold part of the request: let it drain before reuse
          lk.unlock();
          cudaStreamSynchronize(streams[k]);
          lk.lock();
          r->status = st;
          r->done = true;
          r->t_done = Clock::now();
          done_cv.notify_all();
        }
        admitted = true;
      }
      if (!admitted) cv.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
};

extern "C" {

os3d_status os3d_server_default_config(os3d_server_config* c) {
  if (!c) return OS3D_EINVAL;
  c->arena_bytes = (size_t)16 << 30;
  c->max_inflight = 4;
  c->udtype = OS3D_U_C64;
  c->use_graphs = 1;
  c->bank_cache_bytes = (size_t)4 << 30;
  return OS3D_OK;
}

os3d_status os3d_server_create(const os3d_server_config* cfg, const os3d_params* p,
                               os3d_server** out) {
  if (!cfg || !out) return OS3D_EINVAL;
  *out = nullptr;
  if (cfg->arena_bytes < kAlign || cfg->max_inflight < 1 || cfg->max_inflight > 64 ||
      (cfg->udtype != OS3D_U_C64 && cfg->udtype != OS3D_U_BF16X2) ||
      (cfg->use_graphs != 0 && cfg->use_graphs != 1) || cfg->bank_cache_bytes == 0)
    return OS3D_EINVAL;
  auto s = std::make_unique<os3d_server>();
  s->cfg = *cfg;
  if (p) s->params = *p;
  else os3d_default_params(&s->params);
  s->params.overlap = 0;   // concurrency comes from the requests' own streams
  if (cudaGetDevice(&s->dev) != cudaSuccess) return OS3D_ECUDA;
  if (cudaMalloc(&s->arena_base, cfg->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    return OS3D_ENOMEM;
  }
  s->arena = std::make_unique<Arena>(cfg->arena_bytes);
  s->streams.resize(cfg->max_inflight);
  s->slot_req.resize(cfg->max_inflight);
  for (auto& st : s->streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      os3d_server_destroy(s.release());
      return OS3D_ECUDA;
    }
  if (cudaStreamCreateWithFlags(&s->bank_stream, cudaStreamNonBlocking) != cudaSuccess) {
    os3d_server_destroy(s.release());
    return OS3D_ECUDA;
  }
  os3d_server* raw = s.get();
  raw->worker = std::thread([raw] { raw->run(); });
  *out = s.release();
  return OS3D_OK;
}

os3d_status os3d_server_submit(os3d_server* s, const int dims[3], int subdiv, const float* f,
                               float* f_out, long long* ticket) {
  if (!s || !dims || !f || !f_out || !ticket || subdiv < 0 || subdiv > 4) return OS3D_EINVAL;
  auto r = std::make_shared<Request>();
  std::memcpy(r->dims, dims, sizeof(r->dims));
  r->subdiv = subdiv;
  r->f = f;
  r->f_out = f_out;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return OS3D_EINVAL;
    r->id = s->next_id++;
    s->pending.push_back(r);
    s->all[r->id] = r;
    *ticket = r->id;
  }
  s->cv.notify_all();
  return OS3D_OK;
}

os3d_status os3d_server_wait(os3d_server* s, long long ticket, double timeout_s,
                             double* latency_ms) {
  if (!s || timeout_s < 0) return OS3D_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return OS3D_EINVAL;
  std::shared_ptr<Request> r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  if (!s->done_cv.wait_until(lk, deadline, [&] { return r->done; })) return OS3D_ETIMEOUT;
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const os3d_status st = r->status;
  s->all.erase(ticket);
  return st;
}

os3d_status os3d_server_stats(os3d_server* s, long long* completed, long long* graphs_captured,
                              long long* graph_replays) {
  if (!s) return OS3D_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->n_done;
  if (graphs_captured) *graphs_captured = s->n_captured;
  if (graph_replays) *graph_replays = s->n_replayed;
  return OS3D_OK;
}

os3d_status os3d_server_destroy(os3d_server* s) {
  if (!s) return OS3D_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& st : s->streams)
    if (st) cudaStreamSynchronize(st), cudaStreamDestroy(st);
  s->drop_graphs();
  if (s->bank_stream) cudaStreamDestroy(s->bank_stream);
  for (auto& kv : s->banks) os3d_destroy_bank(kv.second.bank);
  if (s->arena_base) cudaFree(s->arena_base);
  delete s;
  return OS3D_OK;
}

}  // extern "C"
