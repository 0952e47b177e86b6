// Serving loop: many beam streams of different channel counts, DM ranges and
// block lengths share one GPU with continuous batching.
//
// Each stream is a beam of the engine, opened when its first block has arrived
// and its device footprint is admitted by the engine's HBM budget (streams
// that do not fit wait until another stream ends and frees its memory), and
// closed after its last block.  The loop, run on the caller's thread:
//   1. completions: a finished batch hands each of its blocks' candidates to
//      the host, stamps the block done, and frees the stream for its next block;
//   2. admission and pushes: every stream whose next block has arrived and
//      whose previous block is done pushes it on the stream's own CUDA stream
//      (the host-to-device copy overlaps the batches already on the GPU);
//   3. one batched launch (tp_run_ready) covers every block pushed in step 2,
//      whatever its channel count, DM range or block length;
// so blocks that arrive while others are on the GPU join the next batch as
// soon as their stream is free, without waiting for a queue to drain.
// Latency of a block = candidates on the host - arrival, on the server clock.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>
#include <vector>

#include "tp_common.cuh"

namespace tp {
int set_error(int code, const char* fmt, ...);
}
using namespace tp;

namespace {

struct Request {
  int stream = -1, seq = 0;
  const void* buf = nullptr;
  int nsamp = 0;
  double arrival = 0, start = -1, done = -1;
  int64_t ncand = 0;
  int status = 0;
  std::vector<tp_candidate> cands;
};

struct StreamState {
  tp_stream_desc desc{};
  std::vector<double> dms;
  tp_plan* plan = nullptr;
  int beam = -1;
  cudaStream_t cs = nullptr;
  std::vector<int> queue;  // request ids, in submission order
  size_t next = 0;         // next request to push
  bool busy = false;       // a block is on the GPU
  bool ended = false;
};

struct Batch {
  cudaEvent_t ev = nullptr;
  std::vector<int> reqs;
};

}  // namespace

struct tp_server {
  tp_engine* e = nullptr;
  tp_rfi_params rfi{};
  double nsigma = 5.0;
  int keep_candidates = 0;
  std::vector<StreamState> streams;
  std::vector<Request> reqs;
  std::vector<Batch> inflight;
  std::vector<tp_plan*> plans;
  std::chrono::steady_clock::time_point t0;
  bool started = false;
  std::vector<tp_candidate> scratch;
};

namespace {

double now_s(const tp_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

bool same_plan(const tp_stream_desc& a, const std::vector<double>& da, const tp_stream_desc& b,
               const std::vector<double>& db) {
  return a.nchan == b.nchan && a.f_lo_mhz == b.f_lo_mhz && a.bw_mhz == b.bw_mhz && a.t_samp_s == b.t_samp_s &&
         a.dtype == b.dtype && da == db;
}

int close_stream(tp_server* s, StreamState& st) {
  if (st.beam >= 0) {
    int rc = tp_beam_close(s->e, st.beam);
    if (rc) return rc;
    st.beam = -1;
  }
  if (st.cs) {
    cudaStreamDestroy(st.cs);
    st.cs = nullptr;
  }
  return TP_OK;
}

}  // namespace

extern "C" {

int tp_server_create(tp_engine* e, const tp_rfi_params* rfi, double nsigma, int keep_candidates, tp_server** out) {
  TP_NVTX_RANGE();
  if (!e || !out) return set_error(TP_EINVAL, "engine or out is NULL");
  tp_server* s = new tp_server();
  s->e = e;
  if (rfi) s->rfi = *rfi;
  else tp_rfi_defaults(&s->rfi);
  s->nsigma = nsigma;
  s->keep_candidates = keep_candidates;
  *out = s;
  return TP_OK;
}

int tp_server_add_stream(tp_server* s, const tp_stream_desc* d, int* stream_id) {
  if (!s || !d || !stream_id || !d->dm_list || d->ndm <= 0) return set_error(TP_EINVAL, "bad stream description");
  if (d->block_nsamp <= 0 || d->cand_capacity <= 0) return set_error(TP_EINVAL, "bad block length / capacity");
  StreamState st;
  st.desc = *d;
  st.dms.assign(d->dm_list, d->dm_list + d->ndm);
  st.desc.dm_list = nullptr;
  // plans are shared by streams with the same band, sampling, DM list and format
  for (size_t i = 0; i < s->streams.size() && !st.plan; ++i)
    if (same_plan(s->streams[i].desc, s->streams[i].dms, st.desc, st.dms)) st.plan = s->streams[i].plan;
  if (!st.plan) {
    int rc = tp_create_plan(s->e, d->nchan, d->f_lo_mhz, d->bw_mhz, d->t_samp_s, st.dms.data(), d->ndm, d->dtype,
                            &s->rfi, s->nsigma, &st.plan);
    if (rc) return rc;
    s->plans.push_back(st.plan);
  }
  size_t need = 0;
  int rc = tp_beam_footprint(st.plan, d->block_nsamp, d->cand_capacity, &need);
  if (rc) return rc;
  *stream_id = (int)s->streams.size();
  s->streams.push_back(std::move(st));
  return TP_OK;
}

int tp_server_submit(tp_server* s, int stream_id, const void* host_block, int nsamp, double arrival_s) {
  TP_NVTX_RANGE();
  if (!s || stream_id < 0 || stream_id >= (int)s->streams.size()) return set_error(TP_EINVAL, "no stream %d", stream_id);
  StreamState& st = s->streams[stream_id];
  if (st.ended) return set_error(TP_EINVAL, "stream %d has ended", stream_id);
  if (!host_block || nsamp <= 0 || nsamp > st.desc.block_nsamp) return set_error(TP_EINVAL, "bad block");
  if (!st.queue.empty() && arrival_s < s->reqs[st.queue.back()].arrival)
    return set_error(TP_EINVAL, "blocks of a stream must arrive in order");
  Request r;
  r.stream = stream_id;
  r.seq = (int)st.queue.size();
  r.buf = host_block;
  r.nsamp = nsamp;
  r.arrival = arrival_s;
  st.queue.push_back((int)s->reqs.size());
  s->reqs.push_back(std::move(r));
  return (int)s->reqs.size() - 1;
}

int tp_server_end_stream(tp_server* s, int stream_id) {
  if (!s || stream_id < 0 || stream_id >= (int)s->streams.size()) return set_error(TP_EINVAL, "no stream %d", stream_id);
  s->streams[stream_id].ended = true;
  return TP_OK;
}

int tp_server_run(tp_server* s, double time_limit_s) {
  TP_NVTX_RANGE();
  if (!s) return set_error(TP_EINVAL, "server is NULL");
  if (!s->started) {
    s->t0 = std::chrono::steady_clock::now();
    s->started = true;
  }
  tp_engine* e = s->e;
  for (;;) {
    bool progressed = false;
    // 1. completions
    for (size_t bi = 0; bi < s->inflight.size();) {
      Batch& b = s->inflight[bi];
      const cudaError_t q = cudaEventQuery(b.ev);
      if (q == cudaErrorNotReady) {
        ++bi;
        continue;
      }
      if (q != cudaSuccess) return cuda_error(q, "serving batch");
      for (int rid : b.reqs) {
        Request& r = s->reqs[rid];
        StreamState& st = s->streams[r.stream];
        const int cap = st.desc.cand_capacity;
        if ((int)s->scratch.size() < cap) s->scratch.resize(cap);
        int n = 0;
        int rc = tp_get_candidates(e, st.beam, s->scratch.data(), cap, &n);
        r.status = rc;
        if (rc && rc != TP_ETRUNC && rc != TP_EOVERFLOW) return rc;
        r.ncand = n;
        if (s->keep_candidates) r.cands.assign(s->scratch.begin(), s->scratch.begin() + std::min(n, cap));
        r.done = now_s(s);
        st.busy = false;
        if (st.ended && st.next >= st.queue.size()) {
          rc = close_stream(s, st);
          if (rc) return rc;
        }
      }
      cudaEventDestroy(b.ev);
      s->inflight.erase(s->inflight.begin() + bi);
      progressed = true;
    }
    // 2. admission and pushes, oldest pending block first
    const double now = now_s(s);
    std::vector<int> order;
    for (int i = 0; i < (int)s->streams.size(); ++i) {
      StreamState& st = s->streams[i];
      if (!st.busy && st.next < st.queue.size() && s->reqs[st.queue[st.next]].arrival <= now) order.push_back(i);
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      return s->reqs[s->streams[a].queue[s->streams[a].next]].arrival <
             s->reqs[s->streams[b].queue[s->streams[b].next]].arrival;
    });
    std::vector<int> pushed;
    for (int i : order) {
      StreamState& st = s->streams[i];
      if (st.beam < 0) {
        int beam = -1;
        int rc = tp_beam_open(e, st.plan, st.desc.block_nsamp, st.desc.cand_capacity, &beam);
        if (rc == TP_EADMIT) continue;  // waits for memory; smaller streams may still fit
        if (rc) return rc;
        st.beam = beam;
        cudaError_t ce = cudaStreamCreateWithFlags(&st.cs, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamCreate");
        rc = tp_beam_set_stream(e, beam, st.cs);
        if (rc) return rc;
      }
      Request& r = s->reqs[st.queue[st.next]];
      int rc = tp_push_block(e, st.beam, r.buf, r.nsamp, 0);
      if (rc) return rc;
      r.start = now_s(s);
      st.busy = true;
      st.next++;
      pushed.push_back(st.queue[st.next - 1]);
    }
    // 3. one batch for everything pushed
    if (!pushed.empty()) {
      int rc = tp_run_ready(e, 0, nullptr);
      if (rc) return rc;
      Batch b;
      cudaError_t ce = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
      if (ce != cudaSuccess) return cuda_error(ce, "cudaEventCreate");
      // the batch ran on the engine stream: tp_run_ready recorded each beam's
      // detection event there, so one event on that stream marks the batch
      void* es = nullptr;
      rc = tp_engine_stream(e, &es);
      if (rc) return rc;
      ce = cudaEventRecord(b.ev, static_cast<cudaStream_t>(es));
      if (ce != cudaSuccess) return cuda_error(ce, "cudaEventRecord");
      b.reqs = pushed;
      s->inflight.push_back(std::move(b));
      progressed = true;
    }
    // done?
    bool all_done = s->inflight.empty();
    double next_arrival = INFINITY;
    for (auto& st : s->streams) {
      if (st.next < st.queue.size()) {
        all_done = false;
        next_arrival = std::min(next_arrival, s->reqs[st.queue[st.next]].arrival);
      }
      if (!st.ended) all_done = false;
    }
    if (all_done) return TP_OK;
    bool only_unended_idle = s->inflight.empty();
    for (auto& st : s->streams)
      if (st.next < st.queue.size()) only_unended_idle = false;
    if (only_unended_idle) return TP_OK;  // everything submitted so far is done
    if (now_s(s) > time_limit_s) return set_error(TP_ETIMEOUT, "serving time limit reached");
    if (!progressed) {
      const double wait = std::min(next_arrival - now_s(s), 200e-6);
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
    }
  }
}

int tp_server_results(tp_server* s, tp_serve_result* out, int cap, int* n) {
  if (!s || (cap > 0 && !out)) return set_error(TP_EINVAL, "bad arguments");
  const int nr = (int)s->reqs.size();
  for (int i = 0; i < nr && i < cap; ++i) {
    const Request& r = s->reqs[i];
    out[i].stream = r.stream;
    out[i].seq = r.seq;
    out[i].arrival_s = r.arrival;
    out[i].start_s = r.start;
    out[i].done_s = r.done;
    out[i].n_candidates = r.ncand;
    out[i].status = r.status;
    out[i].reserved = 0;
  }
  if (n) *n = nr;
  return TP_OK;
}

int tp_server_candidates(tp_server* s, int request, tp_candidate* out, int cap, int* n) {
  if (!s || request < 0 || request >= (int)s->reqs.size()) return set_error(TP_EINVAL, "no request %d", request);
  const Request& r = s->reqs[request];
  if (!s->keep_candidates) return set_error(TP_EINVAL, "server does not keep candidates");
  const int k = std::min((int)r.cands.size(), cap);
  if (k > 0) std::memcpy(out, r.cands.data(), sizeof(tp_candidate) * k);
  if (n) *n = (int)r.cands.size();
  return TP_OK;
}

int tp_server_destroy(tp_server* s) {
  TP_NVTX_RANGE();
  if (!s) return TP_OK;
  tp_sync(s->e);
  for (auto& b : s->inflight) cudaEventDestroy(b.ev);
  for (auto& st : s->streams) close_stream(s, st);
  for (tp_plan* p : s->plans) tp_plan_destroy(p);
  delete s;
  return TP_OK;
}

}  // extern "C"
