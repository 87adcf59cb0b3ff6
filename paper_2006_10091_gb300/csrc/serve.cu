// serve.cu -- a continuous-batching request loop for encrypted
// logistic-regression gradient and inference requests over several ring
// sizes (the paper's workers serving requests, Sec. 4; the key holder's
// refresh of Algorithm 1 runs in-process when a request's weights
// have too few limbs left).
//
// One scheduler thread owns every CUDA call.  Each context (one ring size
// class, keys resident in HBM) has `max_inflight` slots, each a context view
// with its own stream and workspace.  The loop repeatedly
//   * retires slots whose wave has finished (event query), frees the
//     requests' device memory and records their completion;
//   * admits pending requests, oldest first: a wave takes the oldest request
//     and every other pending one with the same context, kind, data level and
//     configuration, up to `max_wave`, as far as the HBM budget allows, and
//     runs on a free slot of that context: host-to-device copies of the
//     inputs, one batched call over all the wave's requests (each request a
//     worker), device-to-host copies of the outputs, an event.
// Requests that arrive while waves are running join the next wave as soon as
// a slot and memory are free, and waves of different slots overlap on the
// device.  Each request's residues do not depend on what it was batched with
// (the refresh randomness comes from the request's own id).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "he_ops.h"

namespace he {

using Clock = std::chrono::steady_clock;

struct ServeReq {
  uint64_t id;
  he_request r;
  Clock::time_point t_submit, t_done;
  int status = HE_OK;
  uint32_t out_level = 0;
  double out_scale = 0.0;
  uint64_t* dev = nullptr;
  size_t dev_bytes = 0;
  uint32_t l_out = 0;
};

struct Slot {
  he_ctx* view = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<ServeReq*> reqs;
  size_t ws_grow = 0;  // workspace growth counted at admission
  bool busy = false;
};

// The weights' level below which a request refreshes them first.
static uint32_t req_need(const he_request& r) {
  return std::max<uint32_t>(r.kind == HE_REQ_INFERENCE ? 5 : 6, r.min_w_level);
}

static size_t req_out_limbs(const he_request& r, uint32_t* l_out) {
  const uint32_t need = req_need(r);
  const uint32_t l0 = r.w_level >= need ? r.w_level : r.z_level;  // refreshed to the data's level
  *l_out = r.kind == HE_REQ_INFERENCE ? l0 - 3 : l0 - 5;
  return r.kind == HE_REQ_INFERENCE ? (size_t)r.nZ * *l_out : *l_out;
}

static size_t req_words(const he_request& r, uint32_t n) {
  uint32_t l_out = 0;
  const size_t out_limbs = req_out_limbs(r, &l_out);
  return (size_t)n * 2 * ((size_t)r.nZ * r.z_level + r.w_level + out_limbs);
}

static LrShape req_shape(const he_request& r) {
  const uint32_t need = req_need(r);
  const bool refresh = r.w_level < need;
  return LrShape{refresh ? r.z_level : r.w_level, r.nZ, refresh};
}

// Workspace bytes a slot's view must grow by to run these requests as one wave.
static size_t ws_growth(he_ctx* view, const std::vector<LrShape>& shapes, uint32_t refresh_level) {
  const size_t need = lr_ws_bytes(view, shapes.data(), shapes.size(), refresh_level);
  return need > view->ws.size ? ws_alloc_bytes(need) - view->ws.size : 0;
}

static void ws_release(he_ctx* view) {
  if (!view->ws.ptr) return;
  cudaStreamSynchronize(view->stream);
  cudaFree(view->ws.ptr);
  view->ws.ptr = nullptr;
  view->ws.size = 0;
}

}  // namespace he

struct he_server {
  std::vector<he_ctx*> ctxs;
  std::vector<std::vector<he::Slot>> slots;
  size_t budget = 0, used = 0;
  uint32_t max_wave = 1;
  size_t max_running = 0;  // 0: no global limit
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<he::ServeReq*> pending;   // guarded by mu
  std::vector<he::ServeReq*> finished;  // guarded by mu
  size_t inflight = 0;                  // requests admitted and not finished (guarded by mu)
  size_t peak_used = 0, waves = 0, running = 0, peak_running = 0;  // statistics (guarded by mu)
  uint64_t next_id = 1;
  std::string error;
};

namespace he {

static bool same_wave(const he_request& a, const he_request& b) {
  return a.ctx == b.ctx && a.kind == b.kind && a.z_level == b.z_level && a.z_scale == b.z_scale &&
         a.min_w_level == b.min_w_level &&
         a.w_scale == b.w_scale && memcmp(&a.cfg, &b.cfg, sizeof(he_lr_config)) == 0;
}

// Enqueue one wave on its slot's stream: inputs in, one batched circuit call
// over the wave's requests (each a worker shard), outputs out, buffers freed,
// an event.  The view's workspace grows inside the call if it must; that
// growth was estimated at admission and is settled here against the real size.
static int enqueue_wave(Slot& sl, std::vector<ServeReq*>& wave) {
  he_ctx* c = sl.view;
  const uint32_t n = c->n;
  std::vector<std::vector<he_ct>> Z(wave.size());
  std::vector<he_ct> W(wave.size()), Wout(wave.size());
  std::vector<std::vector<he_ct>> Sout(wave.size());
  std::vector<he_lr_shard> sh(wave.size());
  for (size_t k = 0; k < wave.size(); ++k) {
    ServeReq* q = wave[k];
    const he_request& r = q->r;
    HE_CUDA(cudaMallocAsync((void**)&q->dev, q->dev_bytes, sl.stream));
    uint64_t* p = q->dev;
    const size_t zw = (size_t)2 * r.z_level * n, ww = (size_t)2 * r.w_level * n;
    HE_CUDA(cudaMemcpyAsync(p, r.Z, sizeof(uint64_t) * zw * r.nZ, cudaMemcpyHostToDevice, sl.stream));
    for (uint32_t i = 0; i < r.nZ; ++i) Z[k].push_back(he_ct{p + i * zw, r.z_level, r.z_level, r.z_scale});
    p += zw * r.nZ;
    HE_CUDA(cudaMemcpyAsync(p, r.W, sizeof(uint64_t) * ww, cudaMemcpyHostToDevice, sl.stream));
    W[k] = he_ct{p, r.w_level, r.w_level, r.w_scale};
    p += ww;
    const uint32_t lo = q->l_out;
    if (r.kind == HE_REQ_INFERENCE) {
      for (uint32_t i = 0; i < r.nZ; ++i) Sout[k].push_back(he_ct{p + (size_t)i * 2 * lo * n, 0, lo, 0.0});
    } else {
      Wout[k] = he_ct{p, 0, lo, 0.0};
    }
    sh[k] = he_lr_shard{Z[k].data(), r.nZ, &W[k], r.kind == HE_REQ_INFERENCE ? nullptr : &Wout[k],
                        r.kind == HE_REQ_INFERENCE ? Sout[k].data() : nullptr, r.refresh_cid, r.min_w_level};
  }
  const he_request& r0 = wave[0]->r;
  HE_TRY(lr_entry(c, sh.data(), sh.size(), &r0.cfg, r0.z_level, 0, r0.kind == HE_REQ_INFERENCE));
  for (size_t k = 0; k < wave.size(); ++k) {
    ServeReq* q = wave[k];
    const he_ct& o = q->r.kind == HE_REQ_INFERENCE ? Sout[k][0] : Wout[k];
    q->out_level = o.level;
    q->out_scale = o.scale;
    const size_t words = (size_t)2 * q->l_out * n * (q->r.kind == HE_REQ_INFERENCE ? q->r.nZ : 1);
    HE_CUDA(cudaMemcpyAsync(q->r.out, o.data, sizeof(uint64_t) * words, cudaMemcpyDeviceToHost, sl.stream));
  }
  return HE_OK;
}

static int launch_wave(he_server* s, Slot& sl, std::vector<ServeReq*>& wave) {
  const size_t ws_before = sl.view->ws.size;
  const int rc = enqueue_wave(sl, wave);
  if (rc != HE_OK) {  // the scheduler thread's message, for he_server_last_error
    std::lock_guard<std::mutex> lk(s->mu);
    s->error = he_last_error();
  }
  for (ServeReq* q : wave) {
    q->status = rc;
    if (q->dev) cudaFreeAsync(q->dev, sl.stream);
    q->dev = nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->used = s->used + sl.view->ws.size - ws_before - sl.ws_grow;
    s->peak_used = std::max(s->peak_used, s->used);
    sl.ws_grow = 0;
  }
  sl.reqs = wave;
  sl.busy = true;
  if (rc != HE_OK) return rc;
  HE_CUDA(cudaEventRecord(sl.done, sl.stream));
  return HE_OK;
}

static void finish(he_server* s, std::vector<ServeReq*>& reqs) {
  std::lock_guard<std::mutex> lk(s->mu);
  const auto now = Clock::now();
  s->running -= 1;
  for (ServeReq* q : reqs) {
    q->t_done = now;
    s->used -= q->dev_bytes;
    s->finished.push_back(q);
    --s->inflight;
  }
  reqs.clear();
  s->cv.notify_all();
}

static void scheduler(he_server* s) {
  int dev = s->ctxs[0]->device;
  cudaSetDevice(dev);
  for (;;) {
    bool progress = false;
    // retire finished waves
    for (auto& row : s->slots)
      for (Slot& sl : row)
        if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) {
          finish(s, sl.reqs);
          sl.busy = false;
          progress = true;
        }
    // admit
    std::vector<std::pair<Slot*, std::vector<ServeReq*>>> launches;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->pending.empty()) {
        bool idle = true;
        for (auto& row : s->slots)
          for (Slot& sl : row) idle = idle && !sl.busy;
        if (idle) return;
      }
      std::vector<bool> tried(s->ctxs.size(), false);
      for (size_t pi = 0; pi < s->pending.size();) {
        if (s->max_running && s->running >= s->max_running) break;
        ServeReq* head = s->pending[pi];
        const uint32_t ci = head->r.ctx;
        if (tried[ci]) { ++pi; continue; }
        Slot* free_slot = nullptr;
        for (Slot& sl : s->slots[ci])
          if (!sl.busy) { free_slot = &sl; break; }
        bool claimed = false;
        for (auto& l : launches) claimed = claimed || l.first == free_slot;
        if (!free_slot || claimed) { tried[ci] = true; ++pi; continue; }
        // under memory pressure, idle slots give their workspace back first
        {
          std::vector<LrShape> one{req_shape(head->r)};
          const size_t want = head->dev_bytes + ws_growth(free_slot->view, one, head->r.z_level);
          if (s->used + want > s->budget)
            for (auto& row : s->slots)
              for (Slot& sl : row) {
                bool mine = &sl == free_slot;
                for (auto& l : launches) mine = mine || l.first == &sl;
                if (sl.busy || mine || !sl.view->ws.ptr) continue;
                s->used -= sl.view->ws.size;
                ws_release(sl.view);
              }
        }
        std::vector<ServeReq*> wave;
        std::vector<LrShape> shapes;
        size_t bytes = 0, grow = 0;
        for (size_t k = pi; k < s->pending.size() && wave.size() < s->max_wave;) {
          ServeReq* q = s->pending[k];
          if (!same_wave(q->r, head->r)) { ++k; continue; }
          shapes.push_back(req_shape(q->r));
          size_t g = ws_growth(free_slot->view, shapes, head->r.z_level);
          if (s->used + bytes + q->dev_bytes + g > s->budget && wave.empty() && s->inflight == 0 &&
              free_slot->view->ws.ptr) {
            // nothing runs and the other idle slots gave their workspaces back
            // above: the slot's own goes too, so that only this request is
            // counted (submit refused any request that alone exceeds the budget)
            s->used -= free_slot->view->ws.size;
            ws_release(free_slot->view);
            g = ws_growth(free_slot->view, shapes, head->r.z_level);
          }
          if (s->used + bytes + q->dev_bytes + g > s->budget) {
            shapes.pop_back();
            break;
          }
          bytes += q->dev_bytes;
          grow = g;
          wave.push_back(q);
          s->pending.erase(s->pending.begin() + k);
        }
        tried[ci] = true;
        if (wave.empty()) continue;
        free_slot->ws_grow = grow;
        s->used += bytes + grow;
        s->peak_used = std::max(s->peak_used, s->used);
        s->inflight += wave.size();
        s->waves += 1;
        s->running += 1;
        s->peak_running = std::max(s->peak_running, s->running);
        launches.push_back({free_slot, wave});
        progress = true;
      }
    }
    for (auto& l : launches) {
      Slot& sl = *l.first;
      if (launch_wave(s, sl, l.second) != HE_OK) {  // the wave's requests carry the error
        cudaStreamSynchronize(sl.stream);
        finish(s, sl.reqs);
        sl.busy = false;
      }
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace he

using namespace he;

extern "C" int he_server_create(const he_server_config* cfg, he_server** out) {
  if (!cfg || !out || !cfg->ctxs || cfg->n_ctx == 0) return fail(HE_EINVAL, "he_server_create: null argument");
  if (cfg->max_inflight < 1 || cfg->max_inflight > 16 || cfg->max_wave < 1)
    return fail(HE_EINVAL, "he_server_create: max_inflight in [1, 16], max_wave >= 1");
  he_server* s = new he_server();
  s->budget = cfg->hbm_budget;
  s->max_wave = cfg->max_wave;
  s->max_running = cfg->max_running;
  for (size_t i = 0; i < cfg->n_ctx; ++i) {
    he_ctx* c = cfg->ctxs[i];
    if (!c) { delete s; return fail(HE_EINVAL, "he_server_create: null context"); }
    s->ctxs.push_back(c);
    std::vector<Slot> row(cfg->max_inflight);
    for (Slot& sl : row) {
      HE_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
      HE_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
      sl.view = ctx_view(c, sl.stream);
    }
    s->slots.push_back(std::move(row));
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return HE_OK;
}

extern "C" int he_server_submit(he_server* s, const he_request* r, uint64_t* id) {
  if (!s || !r || !id) return fail(HE_EINVAL, "he_server_submit: null argument");
  if (r->ctx >= s->ctxs.size()) return fail(HE_EINVAL, "he_server_submit: context index out of range");
  he_ctx* c = s->ctxs[r->ctx];
  if (r->kind != HE_REQ_GRADIENT && r->kind != HE_REQ_INFERENCE) return fail(HE_EINVAL, "he_server_submit: bad kind");
  if (!r->Z || !r->W || !r->out || r->nZ == 0) return fail(HE_EINVAL, "he_server_submit: null buffer");
  if (r->z_level < 1 || r->z_level > (uint32_t)c->L || r->w_level < 1 || r->w_level > r->z_level)
    return fail(HE_EINVAL, "he_server_submit: bad levels");
  if (r->z_level < req_need(*r)) return fail(HE_ELEVEL, "he_server_submit: data level below the circuit's depth");
  ServeReq* q = new ServeReq();
  q->r = *r;
  const size_t out_limbs = req_out_limbs(*r, &q->l_out);
  if (r->out_words < (size_t)2 * out_limbs * c->n) {
    delete q;
    return fail(HE_EINVAL, "he_server_submit: output buffer too small");
  }
  q->dev_bytes = sizeof(uint64_t) * req_words(*r, c->n);
  {  // the request alone: its buffers and a slot's workspace for it
    const LrShape sh = req_shape(*r);
    he_ctx* v = s->slots[r->ctx].empty() ? c : s->slots[r->ctx][0].view;
    const size_t alone = q->dev_bytes + ws_alloc_bytes(lr_ws_bytes(v, &sh, 1, r->z_level));
    if (alone > s->budget) {
      delete q;
      return fail(HE_ENOMEM, "he_server_submit: the request alone needs more device memory than the budget");
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->id = s->next_id++;
    q->t_submit = Clock::now();
    s->pending.push_back(q);
  }
  s->cv.notify_all();
  *id = q->id;
  return HE_OK;
}

extern "C" int he_server_poll(he_server* s, he_result* results, size_t cap, size_t* n_out) {
  if (!s || (!results && cap) || !n_out) return fail(HE_EINVAL, "he_server_poll: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  size_t n = 0;
  while (n < cap && !s->finished.empty()) {
    ServeReq* q = s->finished.front();
    s->finished.erase(s->finished.begin());
    results[n].id = q->id;
    results[n].status = q->status;
    results[n].level = q->out_level;
    results[n].scale = q->out_scale;
    results[n].latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    delete q;
    ++n;
  }
  *n_out = n;
  return HE_OK;
}

extern "C" int he_server_drain(he_server* s, double timeout_s) {
  if (!s) return fail(HE_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                 [&] { return s->pending.empty() && s->inflight == 0; });
  return ok ? HE_OK : fail(HE_ETIMEOUT, "he_server_drain: requests still pending");
}

extern "C" int he_server_stats(he_server* s, size_t* used, size_t* peak_used, size_t* waves,
                               size_t* peak_running) {
  if (!s) return fail(HE_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (used) *used = s->used;
  if (peak_used) *peak_used = s->peak_used;
  if (waves) *waves = s->waves;
  if (peak_running) *peak_running = s->peak_running;
  return HE_OK;
}

extern "C" int he_server_last_error(he_server* s, char* buf, size_t cap) {
  if (!s || !buf || cap == 0) return fail(HE_EINVAL, "he_server_last_error: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  const size_t k = std::min(cap - 1, s->error.size());
  memcpy(buf, s->error.data(), k);
  buf[k] = 0;
  return HE_OK;
}

extern "C" int he_server_destroy(he_server* s) {
  if (!s) return HE_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto& row : s->slots)
    for (Slot& sl : row) {
      ctx_destroy(sl.view);
      cudaEventDestroy(sl.done);
      cudaStreamDestroy(sl.stream);
    }
  for (ServeReq* q : s->pending) delete q;
  for (ServeReq* q : s->finished) delete q;
  delete s;
  return HE_OK;
}
