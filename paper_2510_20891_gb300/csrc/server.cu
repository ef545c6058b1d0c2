// Serving runtime: many datasets' tables resident on one device under a memory
// budget, requests (a dataset and a batch of tracks) admitted as memory frees
// up and evaluated with continuous batching through tfs_eval_batch.
//
// The paper evaluates walker populations in batches (Sec. II.D); serving many
// independent searches at once has no counterpart in the paper.
//
// One worker thread per server owns all device work.  It keeps two batches in
// flight: while one batch runs, arriving requests are admitted (device buffers
// allocated, inputs uploaded on the batch's own stream) and launched as the next
// batch, so the uploads of one batch overlap the kernels of the other.  The
// kernels of all batches run in launch order on one compute stream: the
// statistic kernel holds a whole SM per block, so a later batch's kernel
// started beside an earlier batch's top-k passes would hold those back until it
// ended.  A second thread watches the batches in flight and completes each as
// soon as its last kernel has run, so that neither admission nor completion
// waits on the other.  Admission is FIFO:
// a request waits until its input/output buffers, plus its dataset's table if
// that is not resident, fit under the budget; idle tables (no admitted or
// running request uses them) are evicted least recently used first to make
// room (their bytes are kept in host memory and copied back on the next use).
// Results are copied out by tfs_server_wait in the caller's thread, on one of the
// server's copy streams (one per concurrent waiter).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "tfs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SrvDataset {
  tfs_table* table = nullptr;        // owned; data == nullptr while evicted
  const tfs_basis* basis = nullptr;  // borrowed
  size_t data_bytes = 0, scale_bytes = 0;
  std::vector<unsigned char> host;   // the table's bytes, copied when the dataset is added
  std::vector<float> host_scales;
  bool resident = true;
  bool pooled = false;               // the device copy came from the stream-ordered pool (a reload)
  int pins = 0;                      // admitted or running requests using the table
  int64_t last_use = 0;
  std::vector<int> wsum_m;           // m values whose window sums are counted in the budget
  int64_t wsum_bytes = 0;            // their bytes (built with the first launch that needs them)
  int64_t dev_bytes() const { return (int64_t)(data_bytes + scale_bytes) + wsum_bytes; }
};

enum ReqState { kQueued, kRunning, kDone, kFailed };

struct SrvReq {
  int64_t ticket = 0;
  int ds = 0;
  SrvDataset* dsp = nullptr;       // the dataset (stable: datasets are never moved or freed before the server)
  int64_t N = 0;
  int m = 0, topk = 0, K = 0;
  const double* coeffs = nullptr;  // caller's host memory, read at admission
  const double* f_ref = nullptr;
  void* dev = nullptr;             // one device block: coeffs, f_ref, stat, top-k
  size_t dev_bytes = 0;
  double* d_c = nullptr;
  double* d_f = nullptr;
  float* d_stat = nullptr;
  int64_t* d_ti = nullptr;
  float* d_tv = nullptr;
  Clock::time_point t_submit;
  ReqState state = kQueued;
  int rc = TFS_OK;
  std::string err;
};

// A stream on which tfs_server_wait copies a request's results into the caller's memory
// (all of them enqueued, then one synchronisation).
struct CopySlot {
  cudaStream_t st = nullptr;
};

struct SrvBatch {
  cudaStream_t st = nullptr;     // allocations, table reloads and uploads
  cudaEvent_t up = nullptr;      // the uploads are done
  cudaEvent_t ev = nullptr;      // the batch's last kernel and status copy are done
  int* d_status = nullptr;
  int* h_status = nullptr;  // pinned
  std::vector<SrvReq*> reqs;
  bool busy = false;
};

}  // namespace

struct tfs_server {
  int device = 0;
  int64_t budget = 0;
  int max_jobs = 64;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<SrvDataset*> ds;
  std::deque<SrvReq*> queue;
  std::unordered_map<int64_t, SrvReq*> reqs;
  int64_t next_ticket = 1;
  int64_t used = 0;  // resident tables + admitted/running/uncollected request buffers
  int64_t use_clock = 0;
  SrvBatch batch[2];
  cudaStream_t cst = nullptr;        // the batches' kernels, in launch order
  std::deque<SrvBatch*> inflight;    // launched batches, oldest first (completed by `completer`)
  std::condition_variable cv_inflight;
  std::thread completer;
  bool stop_completer = false;
  std::mutex copy_mu;                // guards copy_free (slots are created on demand)
  std::vector<CopySlot*> copy_free, copy_all;
  std::thread worker;
  bool stop = false;
  // statistics
  int64_t submitted = 0, completed = 0, failed = 0, tracks_completed = 0;
  int64_t evictions = 0, loads = 0, batches = 0, batch_jobs = 0;
  std::vector<double> lat_ms;
};

namespace tfs {
namespace {

// Keep the table's bytes in host memory (once, when the dataset is added).
int keep_host_copy(SrvDataset* d) {
  tfs_table* t = d->table;
  d->host.resize(d->data_bytes);
  TFS_CUDA(cudaMemcpy(d->host.data(), t->data, d->data_bytes, cudaMemcpyDeviceToHost));
  if (t->scales) {
    d->host_scales.resize((size_t)t->n_seg);
    TFS_CUDA(cudaMemcpy(d->host_scales.data(), t->scales, d->scale_bytes, cudaMemcpyDeviceToHost));
  }
  return TFS_OK;
}

// Free the device copy of an idle table (no request in flight reads it) and its window sums, in
// the order of `st`: a reloaded copy goes back to the pool without waiting for the device; the
// table's first allocation (made when it was built) is freed once with cudaFree.
int evict(SrvDataset* d, cudaStream_t st) {
  tfs_table* t = d->table;
  wsum_free_idle(t, st);
  if (d->pooled) {
    TFS_CUDA(cudaFreeAsync(t->data, st));
    if (t->scales) TFS_CUDA(cudaFreeAsync(t->scales, st));
  } else {
    TFS_CUDA(cudaFree(t->data));
    if (t->scales) TFS_CUDA(cudaFree(t->scales));
  }
  t->data = nullptr;
  t->scales = nullptr;
  d->resident = false;
  return TFS_OK;
}

// Bring an evicted table back from its host copy, in the order of `st` (the copy is never
// written again, so nothing waits for the upload here).
int reload(SrvDataset* d, cudaStream_t st) {
  tfs_table* t = d->table;
  retain_pool_memory();
  TFS_CUDA(cudaMallocAsync(&t->data, d->data_bytes, st));
  TFS_CUDA(cudaMemcpyAsync(t->data, d->host.data(), d->data_bytes, cudaMemcpyHostToDevice, st));
  if (d->scale_bytes) {
    TFS_CUDA(cudaMallocAsync((void**)&t->scales, d->scale_bytes, st));
    TFS_CUDA(cudaMemcpyAsync(t->scales, d->host_scales.data(), d->scale_bytes, cudaMemcpyHostToDevice, st));
  }
  d->pooled = true;
  d->resident = true;
  return TFS_OK;
}

// Evict idle tables, least recently used first, until `need` more bytes fit (keep `keep`).
bool make_room(tfs_server* s, int64_t need, int keep, cudaStream_t st) {
  while (s->used + need > s->budget) {
    SrvDataset* victim = nullptr;
    for (size_t i = 0; i < s->ds.size(); ++i) {
      SrvDataset* d = s->ds[i];
      if ((int)i == keep || !d->resident || d->pins > 0) continue;
      if (!victim || d->last_use < victim->last_use) victim = d;
    }
    if (!victim) return false;
    const int64_t freed = victim->dev_bytes();
    if (evict(victim, st) != TFS_OK) return false;
    s->used -= freed;
    victim->wsum_m.clear();
    victim->wsum_bytes = 0;
    ++s->evictions;
  }
  return true;
}

void finish_batch(tfs_server* s, SrvBatch& b) {
  const cudaError_t e = cudaEventSynchronize(b.ev);
  const int st = (e == cudaSuccess) ? *b.h_status : -1;
  for (SrvReq* r : b.reqs) {
    if (e != cudaSuccess) {
      r->state = kFailed;
      r->rc = TFS_ERR_CUDA;
      r->err = cudaGetErrorString(e);
    } else if (st != 0) {
      r->state = kFailed;
      r->rc = TFS_ERR_TIMEOUT;
      r->err = "a bounded device wait gave up";
    } else {
      r->state = kDone;
    }
    r->dsp->pins -= 1;
  }
  b.reqs.clear();
  b.busy = false;
}

// Admit queued requests into batch b (FIFO, under the budget) and launch them.
void launch(tfs_server* s, SrvBatch& b, std::unique_lock<std::mutex>& lk) {
  std::vector<SrvReq*> adm;
  while (!s->queue.empty() && (int)adm.size() < s->max_jobs) {
    SrvReq* r = s->queue.front();
    SrvDataset* d = r->dsp;
    // the request's buffers, its table if evicted, and the table's window sums for this m if new
    const bool new_w = std::find(d->wsum_m.begin(), d->wsum_m.end(), r->m) == d->wsum_m.end();
    const int64_t w_bytes = new_w ? wsum_bytes(d->table, r->m) : 0;
    const int64_t need = (int64_t)r->dev_bytes + (d->resident ? 0 : d->dev_bytes()) + w_bytes;
    if (s->used + need > s->budget && !make_room(s, need, r->ds, b.st)) break;
    if (!d->resident) {
      const int rc = reload(d, b.st);
      if (rc != TFS_OK) {
        s->queue.pop_front();
        r->state = kFailed;
        r->rc = rc;
        r->err = tfs_last_error();
        s->cv_done.notify_all();
        continue;
      }
      s->used += d->dev_bytes();
      ++s->loads;
    }
    cudaError_t e = cudaMallocAsync(&r->dev, r->dev_bytes, b.st);
    if (e != cudaSuccess) {
      s->queue.pop_front();
      r->state = kFailed;
      r->rc = TFS_ERR_OOM;
      r->err = cudaGetErrorString(e);
      s->cv_done.notify_all();
      continue;
    }
    s->used += (int64_t)r->dev_bytes;
    if (new_w) {
      d->wsum_m.push_back(r->m);
      d->wsum_bytes += w_bytes;
      s->used += w_bytes;
    }
    d->pins += 1;
    d->last_use = ++s->use_clock;
    char* p = static_cast<char*>(r->dev);
    r->d_c = reinterpret_cast<double*>(p);
    p += r256((size_t)r->N * r->K * 8);
    if (r->f_ref) {
      r->d_f = reinterpret_cast<double*>(p);
      p += r256((size_t)r->N * 8);
    }
    r->d_stat = reinterpret_cast<float*>(p);
    p += r256((size_t)r->N * 4);
    if (r->topk > 0) {
      r->d_ti = reinterpret_cast<int64_t*>(p);
      p += r256((size_t)r->topk * 8);
      r->d_tv = reinterpret_cast<float*>(p);
    }
    r->state = kRunning;
    s->queue.pop_front();
    adm.push_back(r);
  }
  if (adm.empty()) return;
  b.reqs = adm;
  b.busy = true;
  ++s->batches;
  s->batch_jobs += (int64_t)adm.size();
  // uploads and the launch run without the lock: submitters and waiters keep going
  lk.unlock();
  std::vector<tfs_job> jobs(adm.size());
  int rc = TFS_OK;
  for (size_t i = 0; i < adm.size() && rc == TFS_OK; ++i) {
    SrvReq* r = adm[i];
    cudaError_t e = cudaMemcpyAsync(r->d_c, r->coeffs, (size_t)r->N * r->K * 8, cudaMemcpyHostToDevice, b.st);
    if (e == cudaSuccess && r->f_ref)
      e = cudaMemcpyAsync(r->d_f, r->f_ref, (size_t)r->N * 8, cudaMemcpyHostToDevice, b.st);
    if (e != cudaSuccess) rc = cuda_fail(e, "request upload");
    // the window sums this launch reads, built here on the batch's stream if new (their first
    // build waits for that stream only, not for the compute stream)
    const float* q = nullptr;
    int qp = 0;
    if (rc == TFS_OK) rc = wsum_get(r->dsp->table, r->m, b.st, &q, &qp);
    tfs_job& j = jobs[i];
    std::memset(&j, 0, sizeof(j));
    j.table = r->dsp->table;
    j.basis = r->dsp->basis;
    j.coeffs = r->d_c;
    j.f_ref = r->d_f;
    j.N = r->N;
    j.m = r->m;
    j.topk = r->topk;
    j.stat = r->d_stat;
    j.top_idx = r->d_ti;
    j.top_val = r->d_tv;
  }
  if (rc == TFS_OK) {
    cudaError_t e = cudaEventRecord(b.up, b.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cst, b.up, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "batch upload event");
  }
  if (rc == TFS_OK) rc = tfs_eval_batch(jobs.data(), (int)jobs.size(), b.d_status, s->cst);
  if (rc == TFS_OK) {
    cudaError_t e = cudaMemcpyAsync(b.h_status, b.d_status, sizeof(int), cudaMemcpyDeviceToHost, s->cst);
    if (e == cudaSuccess) e = cudaEventRecord(b.ev, s->cst);
    if (e != cudaSuccess) rc = cuda_fail(e, "batch completion event");
  }
  const std::string msg = rc == TFS_OK ? std::string() : std::string(tfs_last_error());
  if (rc != TFS_OK) {
    cudaStreamSynchronize(b.st);
    cudaStreamSynchronize(s->cst);
  }
  lk.lock();
  if (rc != TFS_OK) {
    for (SrvReq* r : adm) {
      r->state = kFailed;
      r->rc = rc;
      r->err = msg;
      r->dsp->pins -= 1;
    }
    b.reqs.clear();
    b.busy = false;
    s->cv_done.notify_all();
  }
}

void worker_main(tfs_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (s->stop && s->queue.empty() && !s->batch[0].busy && !s->batch[1].busy) break;
    bool progressed = false;
    for (SrvBatch& b : s->batch) {
      if (!b.busy && !s->queue.empty()) {
        const size_t before = s->queue.size();
        launch(s, b, lk);
        if (b.busy) {
          s->inflight.push_back(&b);
          s->cv_inflight.notify_one();
        }
        progressed = progressed || s->queue.size() != before;
      }
    }
    // submissions, completions, collected results and shutdown all notify cv_work
    if (!progressed) s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
  }
}

// Completes batches as their events fire, whichever of the batches in flight ends first.  It polls
// the events of a snapshot of the batches in flight without the lock (only this thread finishes a
// batch, and a batch's event is recorded again only after it has been finished), taking the lock
// again every 50 us to pick up batches launched meanwhile.
void completer_main(tfs_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    while (s->inflight.empty() && !s->stop_completer) s->cv_inflight.wait(lk);
    if (s->inflight.empty()) break;
    const std::vector<SrvBatch*> v(s->inflight.begin(), s->inflight.end());
    lk.unlock();
    SrvBatch* done = nullptr;
    const auto t0 = Clock::now();
    while (!done && Clock::now() - t0 < std::chrono::microseconds(50)) {
      for (SrvBatch* b : v)
        if (cudaEventQuery(b->ev) != cudaErrorNotReady) {
          done = b;
          break;
        }
      if (!done) std::this_thread::yield();
    }
    lk.lock();
    if (!done) continue;
    finish_batch(s, *done);
    s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), done));
    s->cv_done.notify_all();
    s->cv_work.notify_one();
  }
}

}  // namespace
}  // namespace tfs

using namespace tfs;

extern "C" {

int tfs_server_create(int64_t budget_bytes, int max_batch_jobs, tfs_server** out) {
  clear_error();
  TFS_CHECK(out, TFS_ERR_INVALID_ARG, "null output");
  TFS_CHECK(budget_bytes > 0, TFS_ERR_INVALID_ARG, "budget must be positive");
  TFS_CHECK(max_batch_jobs >= 1 && max_batch_jobs <= 4096, TFS_ERR_INVALID_ARG, "max_batch_jobs must be in [1, 4096]");
  int dev = 0;
  TFS_CUDA(cudaGetDevice(&dev));
  tfs_server* s = new tfs_server();
  s->device = dev;
  s->budget = budget_bytes;
  s->max_jobs = max_batch_jobs;
  {
    const cudaError_t e = cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      tfs_server_free(s);
      return cuda_fail(e, "server set-up");
    }
  }
  for (SrvBatch& b : s->batch) {
    cudaError_t e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.up, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_status, sizeof(int));
    if (e != cudaSuccess) {
      tfs_server_free(s);
      return cuda_fail(e, "server set-up");
    }
  }
  s->worker = std::thread(worker_main, s);
  s->completer = std::thread(completer_main, s);
  *out = s;
  return TFS_OK;
}

int tfs_server_add_dataset(tfs_server* s, tfs_table* table, const tfs_basis* basis, int* ds_id) {
  clear_error();
  TFS_CHECK(s && table && basis && ds_id, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(basis->n_seg == table->n_seg, TFS_ERR_INVALID_ARG, "basis and table segment counts differ");
  TFS_CHECK(table->data, TFS_ERR_INVALID_ARG, "table has no device data");
  TFS_CHECK(table->owns, TFS_ERR_INVALID_ARG, "a table view cannot be handed to a server");
  std::lock_guard<std::mutex> lk(s->mu);
  wsum_free(table);  // window sums come back within the budget, as launches need them
  SrvDataset* d = new SrvDataset();
  d->table = table;
  d->basis = basis;
  d->data_bytes = (size_t)table->n_seg * table->row_stride * esize_of(table->dtype);
  d->scale_bytes = table->scales ? (size_t)table->n_seg * sizeof(float) : 0;
  const int rc = keep_host_copy(d);
  if (rc != TFS_OK) {
    delete d;
    return rc;
  }
  d->last_use = ++s->use_clock;
  s->ds.push_back(d);
  s->used += d->dev_bytes();
  *ds_id = (int)s->ds.size() - 1;
  // over budget: evict idle tables, least recently used first (possibly an older one)
  if (s->used > s->budget) make_room(s, 0, -1, s->batch[0].st);
  return TFS_OK;
}

int tfs_server_submit(tfs_server* s, int ds_id, const double* coeffs, const double* f_ref, int64_t N, int m,
                      int topk, int64_t* ticket) {
  clear_error();
  TFS_CHECK(s && coeffs && ticket, TFS_ERR_INVALID_ARG, "null argument");
  TFS_CHECK(N >= 1 && N < ((int64_t)1 << 31), TFS_ERR_INVALID_ARG, "N must be in [1, 2^31)");
  TFS_CHECK(m >= 0 && m <= 64, TFS_ERR_INVALID_ARG, "m must be in [0, 64]");
  TFS_CHECK(topk >= 0 && topk <= 1024, TFS_ERR_INVALID_ARG, "topk must be in [0, 1024]");
  std::lock_guard<std::mutex> lk(s->mu);
  TFS_CHECK(ds_id >= 0 && ds_id < (int)s->ds.size(), TFS_ERR_NOT_FOUND, "unknown dataset %d", ds_id);
  SrvDataset* d = s->ds[ds_id];
  SrvReq* r = new SrvReq();
  r->ds = ds_id;
  r->dsp = d;
  r->N = N;
  r->m = m;
  r->topk = (int)std::min<int64_t>(topk, N);
  r->K = d->basis->K;
  r->coeffs = coeffs;
  r->f_ref = f_ref;
  r->dev_bytes = r256((size_t)N * r->K * 8) + (f_ref ? r256((size_t)N * 8) : 0) + r256((size_t)N * 4) +
                 (r->topk ? r256((size_t)r->topk * 8) + r256((size_t)r->topk * 4) : 0) +
                 (r->topk ? r256(topk_workspace_bytes(N)) : 0) + 4096;
  const int64_t with_table = (int64_t)r->dev_bytes + (int64_t)(d->data_bytes + d->scale_bytes) +
                             wsum_bytes(d->table, m);
  if (with_table > s->budget) {
    delete r;
    set_error("request needs %lld bytes with its table and window sums, over the %lld-byte budget",
              (long long)with_table, (long long)s->budget);
    return TFS_ERR_OOM;
  }
  r->ticket = s->next_ticket++;
  r->t_submit = Clock::now();
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  ++s->submitted;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return TFS_OK;
}

namespace {

cudaError_t take_copy_slot(tfs_server* s, CopySlot** out) {
  {
    std::lock_guard<std::mutex> g(s->copy_mu);
    if (!s->copy_free.empty()) {
      *out = s->copy_free.back();
      s->copy_free.pop_back();
      return cudaSuccess;
    }
  }
  CopySlot* c = new CopySlot();
  cudaError_t e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return e;
  }
  std::lock_guard<std::mutex> g(s->copy_mu);
  s->copy_all.push_back(c);
  *out = c;
  return cudaSuccess;
}

void give_copy_slot(tfs_server* s, CopySlot* c) {
  std::lock_guard<std::mutex> g(s->copy_mu);
  s->copy_free.push_back(c);
}

}  // namespace

int tfs_server_wait(tfs_server* s, int64_t ticket, int timeout_ms, float* stat, int64_t* top_idx, float* top_val) {
  clear_error();
  TFS_CHECK(s, TFS_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  TFS_CHECK(it != s->reqs.end(), TFS_ERR_NOT_FOUND, "unknown ticket %lld", (long long)ticket);
  SrvReq* r = it->second;
  const auto ready = [&] { return r->state == kDone || r->state == kFailed; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    set_error("ticket %lld not finished within %d ms", (long long)ticket, timeout_ms);
    return TFS_ERR_TIMEOUT;
  }
  s->reqs.erase(it);
  lk.unlock();
  int rc = r->rc;
  std::string err = r->err;
  if (r->state == kDone) {
    // copy the results out on a copy slot's stream (the worker's streams keep running)
    cudaSetDevice(s->device);
    CopySlot* c = nullptr;
    cudaError_t e = take_copy_slot(s, &c);
    // Touch the destination's pages first: a device write into pageable pages that were never
    // touched waits on page faults served one by one (about 1 ms for 4 MB of fresh memory, far
    // more with several copies at once); a store per 4 KB maps them on the host beforehand.
    if (stat)
      for (size_t o = 0; o < (size_t)r->N * 4; o += 4096) reinterpret_cast<volatile char*>(stat)[o] = 0;
    if (e == cudaSuccess && stat)
      e = cudaMemcpyAsync(stat, r->d_stat, (size_t)r->N * 4, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && r->topk && top_idx)
      e = cudaMemcpyAsync(top_idx, r->d_ti, (size_t)r->topk * 8, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && r->topk && top_val)
      e = cudaMemcpyAsync(top_val, r->d_tv, (size_t)r->topk * 4, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (c) {
      if (e == cudaSuccess) e = cudaFreeAsync(r->dev, c->st);
      else cudaFree(r->dev);
      give_copy_slot(s, c);
    } else if (r->dev) {
      cudaFree(r->dev);
    }
    if (e != cudaSuccess) {
      rc = TFS_ERR_CUDA;
      err = cudaGetErrorString(e);
    }
  } else if (r->dev) {
    cudaFree(r->dev);
  }
  const double ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
  lk.lock();
  s->used -= (int64_t)r->dev_bytes * (r->dev ? 1 : 0);
  if (rc == TFS_OK) {
    ++s->completed;
    s->tracks_completed += r->N;
    s->lat_ms.push_back(ms);
  } else {
    ++s->failed;
  }
  s->cv_work.notify_one();
  lk.unlock();
  delete r;
  if (rc != TFS_OK) set_error("%s", err.c_str());
  return rc;
}

int tfs_server_get_stats(tfs_server* s, tfs_server_stats* out) {
  clear_error();
  TFS_CHECK(s && out, TFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->tracks_completed = s->tracks_completed;
  out->evictions = s->evictions;
  out->loads = s->loads;
  out->batches = s->batches;
  out->used_bytes = s->used;
  out->budget_bytes = s->budget;
  int64_t res = 0;
  for (SrvDataset* d : s->ds)
    if (d->resident) res += d->dev_bytes();
  out->resident_bytes = res;
  out->mean_jobs_per_batch = s->batches ? (double)s->batch_jobs / (double)s->batches : 0.0;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    const auto q = [&](double p) {
      const size_t i = (size_t)std::min<double>((double)v.size() - 1, std::ceil(p * (double)v.size()) - 1.0);
      return v[i];
    };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    double sum = 0.0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
  }
  return TFS_OK;
}

int tfs_server_free(tfs_server* s) {
  if (!s) return TFS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_completer = true;
    s->cv_inflight.notify_all();
  }
  if (s->completer.joinable()) s->completer.join();
  for (auto& kv : s->reqs) {
    if (kv.second->dev) cudaFree(kv.second->dev);
    delete kv.second;
  }
  cudaDeviceSynchronize();
  for (SrvDataset* d : s->ds) {
    if (d->pooled && d->table->data) {  // a reloaded copy goes back to the pool
      cudaFreeAsync(d->table->data, 0);
      if (d->table->scales) cudaFreeAsync(d->table->scales, 0);
      d->table->data = nullptr;
      d->table->scales = nullptr;
    }
    tfs_table_free(d->table);
    delete d;
  }
  for (CopySlot* c : s->copy_all) {
    cudaStreamSynchronize(c->st);
    cudaStreamDestroy(c->st);
    delete c;
  }
  if (s->cst) {
    cudaStreamSynchronize(s->cst);
    cudaStreamDestroy(s->cst);
  }
  for (SrvBatch& b : s->batch) {
    if (b.ev) cudaEventDestroy(b.ev);
    if (b.st) cudaStreamDestroy(b.st);
    if (b.up) cudaEventDestroy(b.up);
    if (b.d_status) cudaFree(b.d_status);
    if (b.h_status) cudaFreeHost(b.h_status);
  }
  delete s;
  return TFS_OK;
}

}  // extern "C"
