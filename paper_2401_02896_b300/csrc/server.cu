// Frame server: continuous batching of render requests over several CUDA
// streams, with admission against a device-memory budget.
//
// Each worker thread owns a CUDA stream and an internal context (its own
// grow-only frame buffers, events and counters), takes the oldest queued
// request together with later queued requests of the same data set, table,
// transfer function and options (up to max_batch frames), renders them with
// one launch of the render kernel whose work queue spans all their rays (the
// kernels of sphdvr_render_batch), and marks them done once its stream has
// drained.  Frames of different workers overlap on the GPU as well: the
// persistent render kernel of one batch fills the SMs that another's leaves
// idle at its tail.
//
// Memory: the bytes all workers hold stay within the budget.  Before a frame
// grows a worker's buffers the worker checks the budget; when the frame does
// not fit beside what the other workers hold, the worker frees all it holds
// and waits (holding nothing, so waits cannot form a cycle) until the others
// have released enough; workers release their buffers after a request while
// another worker is waiting.  A frame that alone exceeds the budget fails with
// SPHDVR_EBUSY; a batch that does not fit is split into single frames.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sphdvr_internal.h"

namespace sphdvr {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  RenderArgs a{};
  sphdvr_render_opts opts{};
  bool has_opts = false;
  std::vector<float4> tf;
  Clock::time_point t_submit, t_done;
  bool done = false;
  sphdvr_status status = SPHDVR_OK;
  std::string msg;
};

struct Worker;

}  // namespace
}  // namespace sphdvr

struct sphdvr_server {
  sphdvr_ctx* ctx = nullptr;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_mem;
  std::deque<sphdvr::Request*> queue;
  std::unordered_map<uint64_t, sphdvr::Request*> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<sphdvr::Worker*> workers;
  int max_batch = SPHDVR_MAX_BATCH;  // frames one render launch may take
  int64_t max_batch_rays = 512 * 512;  // rays of a batch beyond its first frame's
  int64_t launches = 0, batch_frames = 0, largest_batch = 0;
  size_t held_total = 0;  // device bytes all workers hold
  int waiting_mem = 0;
  // statistics of completed requests
  std::vector<double> lat_ms;
  double rays_done = 0.0;
  bool have_t0 = false;
  sphdvr::Clock::time_point t_first, t_last;
  int64_t completed = 0, failed = 0;
};

namespace sphdvr {
namespace {

struct Worker {
  sphdvr_server* S = nullptr;
  sphdvr_ctx* wctx = nullptr;
  cudaStream_t st = nullptr;
  std::thread th;
  size_t held = 0;          // bytes this worker holds (counted in S->held_total)
  size_t need_now = 0;      // bytes the current frames need in total (set by the sizer)
  bool retry = false;       // the sizer found no room beside the other workers
  bool split = false;       // the batch alone exceeds the budget
  bool fresh = false;       // the worker held no buffers when the current attempt began
  int batch_n = 1;          // frames of the current launch
};

// Update this worker's share of held_total (caller holds S->mu).
void account(Worker* w) {
  const size_t h = ctx_held_bytes(w->wctx);
  w->S->held_total = w->S->held_total - w->held + h;
  w->held = h;
}

void release(Worker* w) {  // caller holds S->mu
  ctx_release_buffers(w->wctx);
  account(w);
  w->S->cv_mem.notify_all();
}

// Reserve `bytes` as this worker's holding (caller holds S->mu).
void reserve(Worker* w, size_t bytes) {
  w->S->held_total = w->S->held_total - w->held + bytes;
  w->held = bytes;
}

// Wait, holding nothing, until `want` bytes fit beside the other workers'
// holdings (caller holds the lock).
void wait_for_room(Worker* w, std::unique_lock<std::mutex>& lk, size_t want) {
  sphdvr_server* S = w->S;
  release(w);
  ++S->waiting_mem;
  S->cv_work.notify_all();  // idle workers release what they hold
  S->cv_mem.wait(lk, [&] { return S->held_total + want <= S->budget || S->stop; });
  --S->waiting_mem;
}

size_t with_headroom(size_t b) { return b + b / 4 + 4096; }

// Pair-buffer sizer used inside a frame: grows the worker's buffers only when
// the result fits the budget beside the other workers' holdings.
sphdvr_status server_sizer(sphdvr_ctx* ctx, FrameWork& fw, size_t pairs, void* user) {
  Worker* w = (Worker*)user;
  sphdvr_server* S = w->S;
  std::unique_lock<std::mutex> lk(S->mu);
  const size_t after = held_after_pair_sizer(ctx, pairs);
  w->need_now = std::max(w->need_now, after);
  if (after > S->budget) {
    if (!w->fresh) {  // buffers of earlier frames count: drop them all and redo the frames
      w->retry = true;
      w->need_now = 0;
      return SPHDVR_EBUSY;
    }
    if (w->batch_n > 1) {
      w->split = true;
      return SPHDVR_EBUSY;
    }
    return set_err(ctx, SPHDVR_EBUSY, "frame needs more device memory than the budget");
  }
  if (S->held_total - w->held + after > S->budget) {
    w->retry = true;
    return SPHDVR_EBUSY;
  }
  reserve(w, std::max(after, w->held));
  lk.unlock();
  sphdvr_status s = ctx_pair_sizer(ctx, fw, pairs, nullptr);
  lk.lock();
  account(w);
  return s;
}

RenderArgs args_of(Request* r) {
  RenderArgs a = r->a;
  a.tf_host = r->tf.data();
  a.opts = r->has_opts ? &r->opts : nullptr;
  return a;
}

// Requests that one launch can render together.
bool same_launch(const Request* x, const Request* y) {
  if (x->a.ds != y->a.ds || x->a.lut != y->a.lut || x->a.tf_n != y->a.tf_n || x->a.tf_lo != y->a.tf_lo ||
      x->a.tf_hi != y->a.tf_hi || x->has_opts != y->has_opts)
    return false;
  if (std::memcmp(x->tf.data(), y->tf.data(), x->tf.size() * sizeof(float4)) != 0) return false;
  if (!x->has_opts) return true;
  const sphdvr_render_opts &a = x->opts, &b = y->opts;
  return a.precision == b.precision && a.anchor_every == b.anchor_every && a.window_h == b.window_h &&
         a.ert_eps == b.ert_eps && a.persistent == b.persistent && a.reinit_dt == b.reinit_dt &&
         a.quant_tau == b.quant_tau && a.quant_sigma == b.quant_sigma;
}

// Render the requests `rs` with one launch and complete them.
void run_batch(Worker* w, std::vector<Request*>& rs) {
  sphdvr_server* S = w->S;
  sphdvr_status s = SPHDVR_OK;
  std::string msg;
  RenderArgs a[SPHDVR_MAX_BATCH];
  w->need_now = 0;
  for (int attempt = 0;; ++attempt) {
    const int n = (int)rs.size();
    for (int f = 0; f < n; ++f) a[f] = args_of(rs[f]);
    w->batch_n = n;
    const size_t fixed = with_headroom(batch_fixed_bytes(w->wctx, a, n));
    {
      std::unique_lock<std::mutex> lk(S->mu);
      w->fresh = ctx_held_bytes(w->wctx) == 0;
      if (fixed > S->budget && n == 1) {
        msg = "frame needs more device memory than the budget";
        s = SPHDVR_EBUSY;
        break;
      }
      if (fixed > S->budget) {
        w->split = true;
      } else {
        const size_t want = std::max(w->held, std::max(fixed, w->need_now));
        if (S->held_total - w->held + want > S->budget) wait_for_room(w, lk, std::max(fixed, w->need_now));
        reserve(w, std::max(w->held, std::max(fixed, w->need_now)));
      }
    }
    if (!w->split) {
      w->retry = false;
      w->wctx->last_error.clear();
      s = render_batch_sized(w->wctx, a, n, w->st, server_sizer, w);
      if (s == SPHDVR_OK) {
        cudaError_t e = cudaStreamSynchronize(w->st);
        if (e != cudaSuccess) s = cuda_err(w->wctx, e, "server frame");
      }
    }
    if (w->split) {
      // the batch does not fit the budget as a whole: put all but the oldest
      // request back at the head of the queue and render that one alone
      cudaStreamSynchronize(w->st);
      std::unique_lock<std::mutex> lk(S->mu);
      for (int f = n - 1; f >= 1; --f) S->queue.push_front(rs[f]);
      rs.resize(1);
      w->split = false;
      w->need_now = 0;
      release(w);
      S->cv_work.notify_all();
      continue;
    }
    if (s == SPHDVR_EBUSY && w->retry && attempt < 64 && !S->stop) {
      // no room beside the other workers: free everything, wait for room, redo the frames
      cudaStreamSynchronize(w->st);
      std::unique_lock<std::mutex> lk(S->mu);
      wait_for_room(w, lk, w->need_now);
      continue;
    }
    if (s != SPHDVR_OK) msg = w->wctx->last_error;
    break;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  account(w);
  const auto t_done = Clock::now();
  if (s == SPHDVR_OK) {
    ++S->launches;
    S->batch_frames += (int64_t)rs.size();
    S->largest_batch = std::max<int64_t>(S->largest_batch, (int64_t)rs.size());
  }
  for (Request* r : rs) {
    r->status = s;
    r->msg = msg;
    r->t_done = t_done;
    r->done = true;
    if (s == SPHDVR_OK) {
      ++S->completed;
      S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
      S->rays_done += (double)r->a.cam.width * r->a.cam.height;
      S->t_last = r->t_done;
    } else {
      ++S->failed;
    }
  }
  if (S->waiting_mem > 0) release(w);
  S->cv_done.notify_all();
}

void worker_main(Worker* w) {
  sphdvr_server* S = w->S;
  cudaSetDevice(S->ctx->device);
  for (;;) {
    std::vector<Request*> rs;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || (S->waiting_mem > 0 && w->held > 0); });
      if (S->waiting_mem > 0 && w->held > 0) {
        release(w);  // another worker waits for device memory
        continue;
      }
      if (S->queue.empty()) break;  // stop requested and nothing left
      rs.push_back(S->queue.front());
      S->queue.pop_front();
      // later requests that can share the launch join it, in queue order,
      // while the batch stays within the frame and ray limits
      int64_t rays = (int64_t)rs[0]->a.cam.width * rs[0]->a.cam.height;
      for (auto it = S->queue.begin(); it != S->queue.end() && (int)rs.size() < S->max_batch;) {
        const int64_t r_ = (int64_t)(*it)->a.cam.width * (*it)->a.cam.height;
        if (rays + r_ <= S->max_batch_rays && same_launch(rs[0], *it)) {
          rays += r_;
          rs.push_back(*it);
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    run_batch(w, rs);
  }
}

void destroy_workers(sphdvr_server* S) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_mem.notify_all();
  for (Worker* w : S->workers) {
    if (w->th.joinable()) w->th.join();
  }
  for (Worker* w : S->workers) {
    cudaSetDevice(S->ctx->device);
    if (w->st) cudaStreamDestroy(w->st);
    if (w->wctx) sphdvr_destroy(w->wctx);
    delete w;
  }
  S->workers.clear();
}

}  // namespace
}  // namespace sphdvr

using namespace sphdvr;

extern "C" {

sphdvr_status sphdvr_server_create(sphdvr_ctx* ctx, size_t hbm_budget, int max_inflight, sphdvr_server** out) {
  if (!ctx || !out) return SPHDVR_EINVAL;
  *out = nullptr;
  if (max_inflight < 1 || max_inflight > 8) return set_err(ctx, SPHDVR_EINVAL, "server: max_inflight out of [1, 8]");
  if (hbm_budget == 0) return set_err(ctx, SPHDVR_EINVAL, "server: hbm_budget is 0");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  sphdvr_server* S = new (std::nothrow) sphdvr_server();
  if (!S) return set_err(ctx, SPHDVR_ENOMEM, "server: out of host memory");
  S->ctx = ctx;
  S->budget = hbm_budget;
  for (int i = 0; i < max_inflight; ++i) {
    Worker* w = new (std::nothrow) Worker();
    sphdvr_status s = w ? sphdvr_create(ctx->device, &w->wctx) : SPHDVR_ENOMEM;
    if (s == SPHDVR_OK) {
      e = cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking);
      if (e != cudaSuccess) s = cuda_err(ctx, e, "server stream");
    }
    if (s != SPHDVR_OK) {
      if (w) {
        if (w->wctx) sphdvr_destroy(w->wctx);
        delete w;
      }
      destroy_workers(S);
      delete S;
      return s;
    }
    w->S = S;
    S->workers.push_back(w);
  }
  for (Worker* w : S->workers) w->th = std::thread(worker_main, w);
  *out = S;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_server_submit(sphdvr_server* S, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                   const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                   float* rgba_out, uint64_t* ticket) {
  if (!S) return SPHDVR_EINVAL;
  sphdvr_ctx* ctx = S->ctx;
  if (!rgba_out || !ticket) return set_err(ctx, SPHDVR_EINVAL, "server_submit: NULL argument");
  sphdvr_status s = check_common(ctx, ds, lut);
  if (s != SPHDVR_OK) return s;
  if ((s = check_opts(ctx, opts)) != SPHDVR_OK || (s = reject_shading(ctx, opts, "server")) != SPHDVR_OK) return s;
  Request* r = new (std::nothrow) Request();
  if (!r) return set_err(ctx, SPHDVR_ENOMEM, "server_submit: out of host memory");
  if ((s = check_camera(ctx, cam, &r->a.cam)) != SPHDVR_OK || (s = pack_tf(ctx, tf, r->tf)) != SPHDVR_OK) {
    delete r;
    return s;
  }
  r->a.ds = ds;
  r->a.lut = &lut->d;
  r->a.tf_n = tf->n;
  r->a.tf_lo = (float)tf->lo;
  r->a.tf_hi = (float)tf->hi;
  r->a.out = rgba_out;
  if (opts) {
    r->opts = *opts;
    r->has_opts = true;
  }
  // a frame that can never fit the budget is refused at once
  RenderArgs a = r->a;
  a.tf_host = r->tf.data();
  a.opts = r->has_opts ? &r->opts : nullptr;
  if (frame_fixed_bytes(ctx, a) > S->budget) {
    delete r;
    return set_err(ctx, SPHDVR_EBUSY, "server_submit: frame needs more device memory than the budget");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    delete r;
    return set_err(ctx, SPHDVR_EINVAL, "server_submit: server is shutting down");
  }
  r->ticket = S->next_ticket++;
  r->t_submit = Clock::now();
  if (!S->have_t0) {
    S->t_first = r->t_submit;
    S->have_t0 = true;
  }
  S->reqs[r->ticket] = r;
  S->queue.push_back(r);
  *ticket = r->ticket;
  S->cv_work.notify_one();
  return SPHDVR_OK;
}

sphdvr_status sphdvr_server_wait(sphdvr_server* S, uint64_t ticket, int timeout_ms) {
  if (!S) return SPHDVR_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return set_err(S->ctx, SPHDVR_ENOTFOUND, "server_wait: unknown ticket");
  Request* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return SPHDVR_ETIMEOUT;
  }
  const sphdvr_status s = r->status;
  if (s != SPHDVR_OK) S->ctx->last_error = r->msg;
  S->reqs.erase(it);
  delete r;
  return s;
}

sphdvr_status sphdvr_server_stats(sphdvr_server* S, double out[8]) {
  if (!S || !out) return SPHDVR_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  for (int i = 0; i < 8; ++i) out[i] = 0.0;
  std::vector<double> v = S->lat_ms;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      const double x = p * (v.size() - 1);
      const size_t i = (size_t)x;
      const double f = x - i;
      return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
    };
    out[0] = pct(0.50);
    out[1] = pct(0.99);
    const double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
    out[2] = span > 0 ? S->rays_done / span : 0.0;
    out[6] = v.back();
  }
  out[3] = (double)S->completed;
  out[4] = (double)S->failed;
  out[5] = (double)S->held_total;
  out[7] = (double)S->queue.size();
  return SPHDVR_OK;
}

sphdvr_status sphdvr_server_set_batch(sphdvr_server* S, int max_batch, int64_t max_batch_rays) {
  if (!S) return SPHDVR_EINVAL;
  if (max_batch < 1 || max_batch > SPHDVR_MAX_BATCH)
    return set_err(S->ctx, SPHDVR_EINVAL, "server_set_batch: max_batch out of [1, SPHDVR_MAX_BATCH]");
  if (max_batch_rays < 0) return set_err(S->ctx, SPHDVR_EINVAL, "server_set_batch: max_batch_rays < 0");
  std::lock_guard<std::mutex> lk(S->mu);
  S->max_batch = max_batch;
  S->max_batch_rays = max_batch_rays;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_server_batch_stats(sphdvr_server* S, int64_t out[4]) {
  if (!S || !out) return SPHDVR_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->launches;
  out[1] = S->batch_frames;
  out[2] = S->largest_batch;
  out[3] = 0;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_server_destroy(sphdvr_server* S) {
  if (!S) return SPHDVR_EINVAL;
  destroy_workers(S);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
  return SPHDVR_OK;
}

}  // extern "C"
