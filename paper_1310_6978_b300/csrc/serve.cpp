// serve.cpp -- continuous-batching request loop.
//
// Requests (formula text, domain, count or enumerate) are compiled on the
// submitting thread and queued.  A server thread runs ticks on its own
// stream: it admits queued requests while their device memory fits the
// budget and a slot is free, gives every admitted request a share of the
// tick's units, and evaluates all of them in ONE interpreter launch over a
// work queue of (slot, unit range) items.  Partial counts stay in device
// memory across ticks (one u64 per slot); a count request finishes when its
// last unit has run.  A model list (enumerate) is tick work too: its units
// are counted in the same launch, each into its own per-unit counter; in the
// tick where its last unit is counted, a scan turns those counts into unit
// offsets and one more launch, over every such request of the tick, writes
// the models in ascending order into the request's device buffer.  Requests
// arriving while a tick runs join the next tick.  Two ticks are in flight:
// the server thread enqueues tick k+1 (admission, items, launches) while the
// GPU runs tick k, then completes tick k (its counts and model lists come
// back through double-buffered pinned memory); programs are uploaded on a
// stream of their own from the stream-ordered pool, so no host step waits
// for the GPU except the completion of the older tick.  Every tick is a
// bounded launch: nothing runs forever on the GPU.
//
// Recurring texts.  A count request whose (text, domain) has been submitted
// jit_after times and has at least jit_min_n letters is a family: a
// background thread compiles its specialised count kernel (NVRTC), orders
// the kernel's items longest first and counts once, off the tick loop.  A
// count request of a ready family is admitted without an interpreter
// upload, and its tick counts all its units with one launch of that kernel
// on a side stream, which runs beside the tick's interpreter launch and
// joins the tick before its counts are copied.  Requests admitted before
// the kernel was ready finish on the interpreter.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fbg.h"
#include "kernels.hpp"
#include "program.hpp"

using namespace fbg;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// a (text, domain) of count requests that may get a specialised kernel,
// found by a hash of the two; the text is kept once its compile is queued,
// and a request uses the kernel only when its own text and domain are equal
// to it
struct TextFamily {
  std::string text;
  int k = 1;
  uint64_t submissions = 0;
  bool queued = false;
  bool ready = false;              // prog holds the built kernel (set under the server's lock)
  fbg_program* prog = nullptr;     // specialised count program, owned by the server
  ~TextFamily() { fbg_program_free(prog); }
};

struct Request {
  uint64_t id = 0;
  TextFamily* fam = nullptr;           // the request's family, if its text may be specialised
  bool jit = false;                // counted by the family's specialised kernel
  int mode = FBG_MODE_COUNT;
  uint64_t cap = 0;
  fbg_program* prog = nullptr;
  int slot = -1;
  uint64_t next_unit = 0, nunits = 0;
  uint64_t mem = 0;
  fbg_status status = FBG_EBUSY;
  uint64_t count = 0;
  std::vector<uint64_t> models;
  // model lists: per-unit counts, their exclusive prefix, the model buffer
  // (stream-ordered allocations of the server's stream)
  unsigned long long* d_unit_counts = nullptr;
  unsigned long long* d_offsets = nullptr;
  unsigned long long* d_models = nullptr;
  double submit_s = 0, admit_s = 0, done_s = 0;
  bool done = false;
  ~Request() { fbg_program_free(prog); }
};

}  // namespace

struct fbg_server {
  fbg_server_options opt{};
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<Request*> pending;
  std::deque<uint64_t> completed;                 // finished requests not yet handed out by fbg_server_completed
  std::vector<Request*> active;                   // admitted, not finished
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t outstanding = 0;
  uint64_t mem_used = 0;
  // device state
  cudaStream_t stream = nullptr;
  FbgInterpProg* d_progs = nullptr;               // one descriptor per slot
  FbgInterpProg* h_progs = nullptr;               // pinned staging
  unsigned long long* d_counts = nullptr;         // per-slot partial counts, then the item counter
  // two ticks can be in flight: items and the copy of the counts are double
  // buffered (index = tick number & 1)
  unsigned long long* h_counts_buf[2] = {nullptr, nullptr};   // pinned
  FbgWorkItem* d_items_buf[2] = {nullptr, nullptr};
  FbgWorkItem* h_items_buf[2] = {nullptr, nullptr};           // pinned
  cudaStream_t upload = nullptr;                  // uploads of admitted programs (pageable sources)
  cudaStream_t copies = nullptr;                  // copies of finished model lists to the host
  cudaEvent_t uploaded = nullptr;
  uint64_t item_cap = 0;
  std::vector<int> free_slots;
  FbgSlotOut* d_slot_out = nullptr;               // per-slot outputs of model lists
  FbgSlotOut* h_slot_out = nullptr;               // pinned staging
  FbgWorkItem* d_witems_buf[2] = {nullptr, nullptr};   // items of the write launch (per tick parity)
  FbgWorkItem* h_witems_buf[2] = {nullptr, nullptr};   // pinned
  size_t witem_cap_buf[2] = {0, 0};
  std::vector<FbgWorkItem> h_wvec;
  unsigned long long* d_scan_total = nullptr;     // scan totals (unused: the slot count has it)
  unsigned long long* h_models = nullptr;         // pinned staging of model lists
  size_t h_models_cap = 0;
  // statistics
  std::atomic<uint64_t> ticks{0}, launches{0};
  double busy_s = 0;
  double admit_s = 0, count_s = 0, enum_s = 0;   // server-thread time by activity
  double gpu_s = 0;                               // device time of the ticks' launches (CUDA events)
  // a tick whose launches are enqueued and not yet completed
  struct InFlight {
    std::vector<Request*> finishing;   // requests whose last units run in this tick
    std::vector<Request*> writes;      // model lists whose ordered write runs in this tick
    int buf = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;   // launches begin / end, counts copied
  };
  cudaEvent_t evs[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  uint64_t tick_no = 0;
  std::deque<InFlight> inflight;
  fbg_status fatal = FBG_OK;
  // recurring texts: families by text and domain, the background compile
  // thread and its queue, the side stream of the specialised launches
  std::unordered_map<uint64_t, std::unique_ptr<TextFamily>> families;
  std::deque<TextFamily*> jit_queue;
  std::condition_variable jit_cv;
  std::thread jit_worker;
  uint64_t jit_started = 0, jit_ready = 0, jit_requests = 0;
  double jit_compile_s = 0;
  cudaStream_t jit_stream = nullptr;
  cudaEvent_t jit_fork = nullptr, jit_join = nullptr;

  void run();
  void jit_run();
  bool enqueue_tick();
  void complete_tick();
  fbg_status admit_locked(Request* r);
  void finish(Request* r, fbg_status s);
  void release_device(Request* r);
};

namespace {

constexpr uint64_t kDefaultBudget = 1ull << 30;

uint64_t request_mem(const fbg_program* p, int mode, uint64_t cap) {
  const InterpBuild& b = p->ib[mode == FBG_MODE_COUNT ? 0 : 1];
  uint64_t m = b.code.ins.size() * 8 + b.code.consts.size() * 8 + sizeof(FbgInterpProg) + b.nitems * sizeof(FbgWorkItem);
  if (mode == FBG_MODE_ENUMERATE) m += cap * 8 + b.nunits * 16;
  return m;
}

}  // namespace

void fbg_server::release_device(Request* r) {
  for (unsigned long long** q : {&r->d_unit_counts, &r->d_offsets, &r->d_models}) {
    if (*q) cudaFreeAsync(*q, stream);
    *q = nullptr;
  }
}

void fbg_server::finish(Request* r, fbg_status s) {
  release_device(r);
  // the result (count, model list) is all a poll needs: the program and its
  // device buffers go now, not when the caller releases the request
  fbg_program_free(r->prog);
  r->prog = nullptr;
  r->status = s;
  r->done_s = now_s();
  r->done = true;
  completed.push_back(r->id);
  if (r->slot >= 0) {
    free_slots.push_back(r->slot);
    r->slot = -1;
  }
  mem_used -= std::min(mem_used, r->mem);
  outstanding--;
  done_cv.notify_all();
}

fbg_status fbg_server::admit_locked(Request* r) {
  if (r->fam && r->fam->ready && r->mode == FBG_MODE_COUNT && r->prog->k == r->fam->k &&
      r->prog->text == r->fam->text) {
    // the family's specialised kernel counts all of it in one launch: a slot
    // for its count, no interpreter upload
    r->jit = true;
    r->mem = 64;
    r->admit_s = now_s();
    r->slot = free_slots.back();
    free_slots.pop_back();
    r->nunits = 1;
    r->next_unit = 0;
    mem_used += r->mem;
    active.push_back(r);
    return FBG_OK;
  }
  // upload the interpreter program (its host half was built at submission)
  // on the upload stream, from the stream-ordered pool, freed on the tick
  // stream: nothing here waits for the ticks in flight
  r->prog->alloc_stream = upload;
  r->prog->free_stream = stream;
  fbg_status s = build_interp(r->prog, r->mode == FBG_MODE_COUNT ? 0 : 1);
  if (s != FBG_OK) return s;
  r->mem = request_mem(r->prog, r->mode, r->cap);
  r->admit_s = now_s();
  const bool count = r->mode == FBG_MODE_COUNT;
  const InterpBuild& b = r->prog->ib[count ? 0 : 1];
  if (!count && b.units_per_item != 1) return set_error(FBG_ETOOBIG, "too many units for a model list");
  r->slot = free_slots.back();
  free_slots.pop_back();
  r->nunits = b.live_units();   // positions in the program's list of live units
  r->next_unit = 0;
  FbgInterpProg G = b.code.prog;
  G.ins = b.d_ins;
  G.consts = b.d_consts;
  h_progs[r->slot] = G;
  cudaError_t e = cudaMemcpyAsync(d_progs + r->slot, h_progs + r->slot, sizeof G, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_counts + r->slot, 0, 8, stream);
  if (e == cudaSuccess && !count) {
    // per-unit counts (zeroed), offsets and the model buffer of this request
    const size_t nu = (size_t)b.nunits;
    e = cudaMallocAsync((void**)&r->d_unit_counts, nu * 8, stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&r->d_offsets, nu * 8, stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&r->d_models, std::max<size_t>(1, (size_t)r->cap) * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_unit_counts, 0, nu * 8, stream);
    if (e == cudaSuccess) {
      h_slot_out[r->slot] = FbgSlotOut{r->d_unit_counts, r->d_offsets, r->d_models, r->cap};
      e = cudaMemcpyAsync(d_slot_out + r->slot, h_slot_out + r->slot, sizeof(FbgSlotOut), cudaMemcpyHostToDevice,
                          stream);
    }
  }
  if (e != cudaSuccess) {
    free_slots.push_back(r->slot);
    r->slot = -1;
    release_device(r);
    return cuda_error(e, "server admit");
  }
  mem_used += r->mem;
  active.push_back(r);
  return FBG_OK;
}

// Enqueue one tick: admission, the shared count launch over a share of every
// admitted request with units left, and the scans and ordered write launch
// of the model lists whose last units it counts, then the copy of the slot
// counts into this tick's host buffer.  Nothing waits for the GPU here.
// Returns false when there was nothing to launch.
bool fbg_server::enqueue_tick() {
  double t0 = now_s();
  std::vector<Request*> work;    // interpreter work
  std::vector<Request*> jwork;   // requests counted by their family's specialised kernel
  bool admitted = false;
  {
    std::unique_lock<std::mutex> lk(mu);
    const double ta = now_s();
    // admission by device memory and free slots, in arrival order
    while (!pending.empty()) {
      Request* r = pending.front();
      if (free_slots.empty()) break;
      // estimate before building; a request larger than the whole budget still runs alone
      uint64_t est = (uint64_t)r->prog->g->dag.size() * 64 + (r->mode == FBG_MODE_ENUMERATE ? r->cap * 8 : 0);
      if (mem_used && mem_used + est > opt.mem_budget_bytes) break;
      pending.pop_front();
      fbg_status s = admit_locked(r);
      if (s != FBG_OK) {
        finish(r, s);
      } else if (r->nunits == 0) {
        // the build left no unit that can hold a model (a conjunct over unit
        // letters is false on every one): no models, nothing to launch.  The
        // program's memory is freed on the tick stream, after its upload
        cudaError_t e = cudaEventRecord(uploaded, upload);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, uploaded, 0);
        r->count = 0;
        finish(r, e == cudaSuccess ? FBG_OK : cuda_error(e, "server admit"));
      } else {
        admitted = true;
      }
    }
    active.erase(std::remove_if(active.begin(), active.end(), [](Request* q) { return q->done; }), active.end());
    admit_s += now_s() - ta;
    for (Request* r : active)
      if (r->next_unit < r->nunits) (r->jit ? jwork : work).push_back(r);   // units not yet launched
  }
  if (work.empty() && jwork.empty()) return false;
  const double tc = now_s();
  InFlight f;
  f.buf = (int)(tick_no & 1);
  f.ev0 = evs[f.buf][0];
  f.ev1 = evs[f.buf][1];
  f.ev2 = evs[f.buf][2];
  FbgWorkItem* h_items = h_items_buf[f.buf];
  FbgWorkItem* d_items = d_items_buf[f.buf];
  cudaError_t e = cudaSuccess;
  // the programs admitted above are uploaded on the upload stream
  if (admitted) {
    e = cudaEventRecord(uploaded, upload);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, uploaded, 0);
  }
  // one launch over a share of every admitted request: count requests in
  // runs of up to 8 consecutive live units, model lists one unit per item
  // (each item's count also goes to that unit's counter).  The tick's work
  // is bounded by tick_units units and tick_assignments assignments; the
  // requests with the least remaining work go first and take all of it when
  // it fits their fair share of what is left, the others take a fair share
  // (at least one unit), so short requests finish in the tick they join
  // while long ones keep advancing.
  auto unit_size = [](const Request* r) {
    const InterpBuild& ib = r->prog->ib[r->mode == FBG_MODE_COUNT ? 0 : 1];
    return (1ull << r->prog->n) / std::max<uint64_t>(1, ib.nunits);
  };
  auto remaining = [&](const Request* r) { return (double)(r->nunits - r->next_unit) * (double)unit_size(r); };
  std::stable_sort(work.begin(), work.end(),
                   [&](const Request* x, const Request* y) { return remaining(x) < remaining(y); });
  double assign_left = (double)opt.tick_assignments;
  uint64_t units_left = opt.tick_units;
  uint64_t n = 0;
  unsigned nslots = 1;
  for (size_t wi = 0; wi < work.size(); wi++) {
    Request* r = work[wi];
    if (n >= item_cap || units_left == 0) break;   // the rest waits for the next tick
    const bool cnt = r->mode == FBG_MODE_COUNT;
    const double fair = assign_left / (double)(work.size() - wi);
    const uint64_t usz = std::max<uint64_t>(1, unit_size(r));
    uint64_t take = r->nunits - r->next_unit;
    if ((double)take * (double)usz > fair) take = std::max<uint64_t>(1, (uint64_t)(fair / (double)usz));
    take = std::min<uint64_t>(take, std::max<uint64_t>(1, units_left / (work.size() - wi)));
    take = std::min<uint64_t>(take, r->nunits - r->next_unit);
    assign_left = std::max(0.0, assign_left - (double)take * (double)usz);
    units_left -= std::min(units_left, take);
    const InterpBuild& ib = r->prog->ib[cnt ? 0 : 1];
    uint64_t i = r->next_unit;
    const uint64_t end = r->next_unit + take;
    // runs of consecutive units of at most 2^22 assignments (and 8 units)
    const uint64_t run_max = cnt ? std::max<uint64_t>(1, std::min<uint64_t>(8, (1ull << 22) / usz)) : 1;
    while (i < end && n < item_cap) {
      const uint64_t u0 = ib.unit_at(i);
      uint64_t len = 1;
      while (i + len < end && len < run_max && ib.unit_at(i + len) == u0 + len) len++;
      h_items[n++] = FbgWorkItem{(unsigned)r->slot, cnt ? 0u : FBG_ITEM_UNIT_COUNTS, u0, u0 + len};
      i += len;
    }
    r->next_unit = i;
    nslots = std::max(nslots, ib.code.nslots);
    if (r->next_unit >= r->nunits) {
      f.finishing.push_back(r);
      if (!cnt) f.writes.push_back(r);
    }
  }
  uint64_t slots = (uint64_t)opt.max_inflight;
  if (e == cudaSuccess && n)
    e = cudaMemcpyAsync(d_items, h_items, n * sizeof(FbgWorkItem), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaEventRecord(f.ev0, stream);
  // the specialised counts first, on the side stream (after the slots'
  // zeroing above), so that they run beside the interpreter launch
  fbg_status js = FBG_OK;
  if (e == cudaSuccess && !jwork.empty()) {
    e = cudaEventRecord(jit_fork, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(jit_stream, jit_fork, 0);
    for (Request* r : jwork) {
      if (e != cudaSuccess || js != FBG_OK) break;
      bool used_jit = false;
      js = launch_count(r->fam->prog, jit_stream, d_counts + r->slot, nullptr, &used_jit);
      r->next_unit = r->nunits;
      f.finishing.push_back(r);
      launches++;
    }
    if (e == cudaSuccess) e = cudaEventRecord(jit_join, jit_stream);
    jit_requests += jwork.size();
  }
  FbgLaunch P{};
  P.unit_begin = 0;
  P.unit_end = ~0ull;
  if (e == cudaSuccess && n) {
    e = cudaMemsetAsync(d_counts + slots, 0, 8, stream);
    int per_sm = interp_blocks_per_sm(0, nslots);
    int grid = (int)std::min<uint64_t>(n, (uint64_t)device_sms() * (uint64_t)std::max(1, per_sm));
    if (e == cudaSuccess)
      e = launch_interp(0, d_progs, d_items, n, d_counts + slots, d_counts, nullptr, P, nslots, std::max(1, grid),
                        stream, d_slot_out);
    launches++;
  }
  // model lists complete in this launch: offsets by a scan of the unit
  // counts, then one ordered write launch over all of them
  if (e == cudaSuccess && !f.writes.empty()) {
    h_wvec.clear();
    unsigned wslots = 1;
    for (Request* r : f.writes) {
      const InterpBuild& ib = r->prog->ib[1];
      if (e == cudaSuccess) e = launch_scan(r->d_unit_counts, r->d_offsets, ib.nunits, d_scan_total, stream);
      ib.append_items(h_wvec, (unsigned)r->slot, 0, ib.live_units(), 1);
      wslots = std::max(wslots, ib.code.nslots);
    }
    // the write launch's items, double buffered like the count items: the
    // buffers of this index were last used by the tick before the previous
    // one, which has completed
    const size_t nw = h_wvec.size();
    if (e == cudaSuccess && nw > witem_cap_buf[f.buf]) {
      if (h_witems_buf[f.buf]) cudaFreeHost(h_witems_buf[f.buf]);
      if (d_witems_buf[f.buf]) cudaFreeAsync(d_witems_buf[f.buf], stream);
      h_witems_buf[f.buf] = nullptr;
      d_witems_buf[f.buf] = nullptr;
      witem_cap_buf[f.buf] = 0;
      e = cudaMallocHost((void**)&h_witems_buf[f.buf], nw * sizeof(FbgWorkItem));
      if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_witems_buf[f.buf], nw * sizeof(FbgWorkItem), stream);
      if (e == cudaSuccess) witem_cap_buf[f.buf] = nw;
    }
    FbgWorkItem* d_witems = d_witems_buf[f.buf];
    if (e == cudaSuccess) {
      std::memcpy(h_witems_buf[f.buf], h_wvec.data(), nw * sizeof(FbgWorkItem));
      e = cudaMemcpyAsync(d_witems, h_witems_buf[f.buf], nw * sizeof(FbgWorkItem), cudaMemcpyHostToDevice, stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counts + slots, 0, 8, stream);
    int wper = interp_blocks_per_sm(2, wslots);
    int wgrid = (int)std::min<uint64_t>(h_wvec.size(), (uint64_t)device_sms() * (uint64_t)std::max(1, wper));
    if (e == cudaSuccess)
      e = launch_interp(2, d_progs, d_witems, h_wvec.size(), d_counts + slots, nullptr, nullptr, P, wslots,
                        std::max(1, wgrid), stream, d_slot_out);
    launches += 1 + f.writes.size();
  }
  if (e == cudaSuccess && !jwork.empty()) e = cudaStreamWaitEvent(stream, jit_join, 0);
  if (e == cudaSuccess) e = cudaEventRecord(f.ev1, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_counts_buf[f.buf], d_counts, slots * 8, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaEventRecord(f.ev2, stream);
  if (e != cudaSuccess || js != FBG_OK) {
    if (e != cudaSuccess) cuda_error(e, "server tick");
    std::unique_lock<std::mutex> lk(mu);
    fatal = e != cudaSuccess ? FBG_ECUDA : js;
    for (Request* r : work) finish(r, fatal);
    for (Request* r : jwork) finish(r, fatal);
    active.erase(std::remove_if(active.begin(), active.end(), [](Request* r) { return r->done; }), active.end());
    count_s += now_s() - tc;
    return false;
  }
  inflight.push_back(std::move(f));
  tick_no++;
  count_s += now_s() - tc;
  busy_s += now_s() - t0;
  return true;
}

// Complete the oldest tick in flight: wait for it, copy the model lists it
// wrote to the host, finish the requests whose last units it ran.
void fbg_server::complete_tick() {
  const double t0 = now_s();
  InFlight f = std::move(inflight.front());
  inflight.pop_front();
  // the tick's launches and the copy of its counts are done (the next tick,
  // if enqueued, may still run; it writes the other count buffer)
  cudaError_t e = cudaEventSynchronize(f.ev2);
  if (e == cudaSuccess) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, f.ev0, f.ev1) == cudaSuccess) gpu_s += ms * 1e-3;
  }
  const unsigned long long* hc = h_counts_buf[f.buf];
  const double tw = now_s();
  for (Request* r : f.writes) {
    if (e != cudaSuccess) break;
    const uint64_t written = std::min<uint64_t>(hc[r->slot], r->cap);
    if (written > h_models_cap) {
      if (h_models) cudaFreeHost(h_models);
      h_models = nullptr;
      h_models_cap = 0;
      e = cudaMallocHost((void**)&h_models, written * 8);
      if (e != cudaSuccess) break;
      h_models_cap = written;
    }
    if (written) e = cudaMemcpyAsync(h_models, r->d_models, written * 8, cudaMemcpyDeviceToHost, copies);
    if (e == cudaSuccess) e = cudaStreamSynchronize(copies);
    if (e == cudaSuccess) r->models.assign(h_models, h_models + written);
  }
  enum_s += now_s() - tw;
  std::unique_lock<std::mutex> lk(mu);
  if (e != cudaSuccess) {
    cuda_error(e, "server tick");
    fatal = FBG_ECUDA;
    for (Request* r : f.finishing) finish(r, FBG_ECUDA);
  } else {
    for (Request* r : f.finishing) {
      r->count = hc[r->slot];
      finish(r, FBG_OK);
    }
  }
  active.erase(std::remove_if(active.begin(), active.end(), [](Request* r) { return r->done; }), active.end());
  ticks++;
  busy_s += now_s() - t0;
}

// The background compiles of recurring texts: build the specialised count
// kernel, order its items longest first (one timed launch) and count once on
// a stream of this thread, then publish the program to the tick loop.  A
// failed build leaves the family on the interpreter.
void fbg_server::jit_run() {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    TextFamily* fam = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      jit_cv.wait(lk, [&] { return stop || !jit_queue.empty(); });
      if (stop) break;
      fam = jit_queue.front();
      jit_queue.pop_front();
    }
    const double t0 = now_s();
    fbg_program* p = nullptr;
    fbg_status s = have_stream ? fbg_compile(fam->text.c_str(), fam->k, &p) : FBG_ECUDA;
    if (s == FBG_OK) {
      p->opt_engine = FBG_ENGINE_JIT;
      s = fbg_schedule_units(p, st);
    }
    uint64_t c = 0;
    if (s == FBG_OK) s = fbg_count(p, st, &c);   // leaves the self-resetting counters clean
    std::lock_guard<std::mutex> lk(mu);
    jit_compile_s += now_s() - t0;
    if (s == FBG_OK) {
      fam->prog = p;
      fam->ready = true;
      jit_ready++;
    } else {
      fbg_program_free(p);
    }
  }
  if (st) cudaStreamDestroy(st);
}

// Two ticks in flight: while the GPU runs one, the server thread admits
// requests and enqueues the next, then completes the older one.
void fbg_server::run() {
  cudaSetDevice(device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || !pending.empty() || !active.empty() || !inflight.empty(); });
      if (stop && inflight.empty()) return;
    }
    bool queued = false;
    if (inflight.size() < 2 && !stop) queued = enqueue_tick();
    if (!inflight.empty() && (inflight.size() >= 2 || !queued)) complete_tick();
  }
}

extern "C" {

fbg_status fbg_server_create(const fbg_server_options* opt, fbg_server** out) {
  if (!out) return set_error(FBG_EINVAL, "null argument");
  *out = nullptr;
  auto* s = new fbg_server();
  if (opt) s->opt = *opt;
  if (!s->opt.mem_budget_bytes) s->opt.mem_budget_bytes = kDefaultBudget;
  if (s->opt.max_inflight <= 0) s->opt.max_inflight = 4096;
  if (!s->opt.tick_units) s->opt.tick_units = 65536;
  if (!s->opt.tick_assignments) s->opt.tick_assignments = 1ull << 36;
  if (!s->opt.jit_min_n) s->opt.jit_min_n = 30;
  if (s->opt.jit_after <= 0) s->opt.jit_after = 2;
  if (s->opt.jit_max_programs <= 0) s->opt.jit_max_programs = 64;
  s->item_cap = s->opt.tick_units + 2 * (uint64_t)s->opt.max_inflight + 16;
  cudaGetDevice(&s->device);
  const size_t slots = (size_t)s->opt.max_inflight;
  cudaError_t e;
  bool ev_ok = true;
  for (auto& pair : s->evs)
    for (auto& ev : pair) ev_ok = ev_ok && cudaEventCreate(&ev) == cudaSuccess;
  if (!ev_ok) {
    fbg_server_free(s);
    return set_error(FBG_ECUDA, "server setup: cudaEventCreate");
  }
  if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->copies, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->jit_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->jit_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->jit_join, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->uploaded, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_progs, slots * sizeof(FbgInterpProg))) != cudaSuccess ||
      (e = cudaMallocHost(&s->h_progs, slots * sizeof(FbgInterpProg))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_counts, (slots + 1) * 8)) != cudaSuccess ||
      (e = cudaMallocHost(&s->h_counts_buf[0], slots * 8)) != cudaSuccess ||
      (e = cudaMallocHost(&s->h_counts_buf[1], slots * 8)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_items_buf[0], s->item_cap * sizeof(FbgWorkItem))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_items_buf[1], s->item_cap * sizeof(FbgWorkItem))) != cudaSuccess ||
      (e = cudaMallocHost(&s->h_items_buf[0], s->item_cap * sizeof(FbgWorkItem))) != cudaSuccess ||
      (e = cudaMallocHost(&s->h_items_buf[1], s->item_cap * sizeof(FbgWorkItem))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_slot_out, slots * sizeof(FbgSlotOut))) != cudaSuccess ||
      (e = cudaMallocHost(&s->h_slot_out, slots * sizeof(FbgSlotOut))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_scan_total, 8)) != cudaSuccess) {
    fbg_server_free(s);
    return cuda_error(e, "server setup");
  }
  for (int i = (int)slots - 1; i >= 0; i--) s->free_slots.push_back(i);
  s->worker = std::thread([s] { s->run(); });
  if (s->opt.jit_min_n > 0) s->jit_worker = std::thread([s] { s->jit_run(); });
  *out = s;
  return FBG_OK;
}

fbg_status fbg_server_submit(fbg_server* s, const char* formula, int domain_k, int mode, uint64_t cap,
                             uint64_t* request_id) {
  if (!s || !formula || !request_id || (mode != FBG_MODE_COUNT && mode != FBG_MODE_ENUMERATE))
    return set_error(FBG_EINVAL, "bad argument");
  const double t_submit = now_s();   // a request's latency includes its compile and host build
  fbg_program* p = nullptr;
  fbg_status st = fbg_compile(formula, domain_k, &p);
  if (st != FBG_OK) return st;
  // ticks run the interpreter: no kernel compile on the server thread.  A
  // count is cut into up to 2^20 units (model lists: 2^16, which keeps their
  // per-unit counters small), so that a large request becomes many short
  // work items that spread over every SM; the units on which a conjunct over
  // unit letters is false are left out at build time, and each of the
  // remaining ones prunes letter by letter (one letter per loop level)
  p->opt_engine = FBG_ENGINE_INTERP;
  p->opt_unit_bits = mode == FBG_MODE_COUNT ? 20 : 16;
  // the host half of the interpreter build runs here, on the submitting
  // thread; admission on the server thread then only uploads it
  st = prebuild_interp_host(p, mode == FBG_MODE_COUNT ? 0 : 1);
  if (st != FBG_OK) {
    fbg_program_free(p);
    return st;
  }
  if (p->n > (mode == FBG_MODE_COUNT ? 63 : 40)) {
    fbg_program_free(p);
    return set_error(FBG_ETOOBIG, "request too large");
  }
  auto r = std::make_unique<Request>();
  r->prog = p;
  r->mode = mode;
  r->cap = cap;
  r->submit_s = t_submit;
  const bool may_jit = mode == FBG_MODE_COUNT && s->opt.jit_min_n > 0 && p->n >= s->opt.jit_min_n &&
                       p->g->root != 0 && p->g->root != 1;
  const uint64_t fkey = may_jit ? std::hash<std::string>{}(p->text) ^ (0x9E3779B97F4A7C15ull * (uint64_t)(domain_k + 1))
                                : 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (may_jit) {
      // the family of this (text, domain): count its submissions, queue its
      // compile at the jit_after-th while the server keeps fewer than
      // jit_max_programs
      auto it = s->families.find(fkey);
      if (it == s->families.end()) it = s->families.emplace(fkey, std::make_unique<TextFamily>()).first;
      TextFamily* fam = it->second.get();
      fam->submissions++;
      if (!fam->queued && fam->submissions >= (uint64_t)s->opt.jit_after &&
          s->jit_started < (uint64_t)s->opt.jit_max_programs) {
        fam->text = p->text;
        fam->k = domain_k;
        fam->queued = true;
        s->jit_started++;
        s->jit_queue.push_back(fam);
        s->jit_cv.notify_one();
      }
      r->fam = fam;
    }
    r->id = s->next_id++;
    *request_id = r->id;
    s->pending.push_back(r.get());
    s->outstanding++;
    s->all.emplace(r->id, std::move(r));
  }
  s->cv.notify_one();
  return FBG_OK;
}

fbg_status fbg_server_poll(fbg_server* s, uint64_t id, fbg_result* out) {
  if (!s || !out) return set_error(FBG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return set_error(FBG_EINVAL, "unknown request");
  Request* r = it->second.get();
  if (!r->done) return FBG_EBUSY;
  out->status = r->status;
  out->count = r->count;
  out->written = r->models.size();
  out->models = r->models.empty() ? nullptr : r->models.data();
  out->submit_s = r->submit_s;
  out->admit_s = r->admit_s;
  out->done_s = r->done_s;
  return FBG_OK;
}

fbg_status fbg_server_completed(fbg_server* s, uint64_t* ids, size_t max_ids, size_t* n) {
  if (!s || !n || (max_ids && !ids)) return set_error(FBG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  size_t k = 0;
  while (k < max_ids && !s->completed.empty()) {
    ids[k++] = s->completed.front();
    s->completed.pop_front();
  }
  *n = k;
  return FBG_OK;
}

fbg_status fbg_server_drain(fbg_server* s, double timeout_s) {
  if (!s) return set_error(FBG_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return s->outstanding == 0; };
  if (timeout_s > 0) {
    if (!s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
      return set_error(FBG_ETIMEOUT, "requests still running");
  } else {
    s->done_cv.wait(lk, ready);
  }
  return s->fatal;
}

fbg_status fbg_server_release(fbg_server* s, uint64_t id) {
  if (!s) return set_error(FBG_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end() || !it->second->done) return set_error(FBG_EINVAL, "unknown or unfinished request");
  s->all.erase(it);
  return FBG_OK;
}

fbg_status fbg_server_stats(fbg_server* s, uint64_t* ticks, uint64_t* launches, double* busy_s) {
  if (!s) return set_error(FBG_EINVAL, "null server");
  if (ticks) *ticks = s->ticks.load();
  if (launches) *launches = s->launches.load();
  if (busy_s) *busy_s = s->busy_s;
  return FBG_OK;
}

fbg_status fbg_server_gpu_time(fbg_server* s, double* gpu_s) {
  if (!s || !gpu_s) return set_error(FBG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *gpu_s = s->gpu_s;
  return FBG_OK;
}

fbg_status fbg_server_jit_stats(fbg_server* s, uint64_t* programs, uint64_t* requests, double* compile_s) {
  if (!s) return set_error(FBG_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (programs) *programs = s->jit_ready;
  if (requests) *requests = s->jit_requests;
  if (compile_s) *compile_s = s->jit_compile_s;
  return FBG_OK;
}

fbg_status fbg_server_profile(fbg_server* s, double* admit_s, double* count_s, double* enum_s) {
  if (!s) return set_error(FBG_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (admit_s) *admit_s = s->admit_s;
  if (count_s) *count_s = s->count_s;
  if (enum_s) *enum_s = s->enum_s;
  return FBG_OK;
}

void fbg_server_free(fbg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->jit_cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->jit_worker.joinable()) s->jit_worker.join();
  if (s->jit_stream) cudaStreamSynchronize(s->jit_stream);
  if (s->stream) {
    for (auto& kv : s->all) s->release_device(kv.second.get());
    for (int b = 0; b < 2; b++) {
      if (s->d_witems_buf[b]) cudaFreeAsync(s->d_witems_buf[b], s->stream);
      s->d_witems_buf[b] = nullptr;
    }
    cudaStreamSynchronize(s->stream);
  }
  s->all.clear();
  s->families.clear();
  if (s->jit_fork) cudaEventDestroy(s->jit_fork);
  if (s->jit_join) cudaEventDestroy(s->jit_join);
  if (s->jit_stream) cudaStreamDestroy(s->jit_stream);
  if (s->d_progs) cudaFree(s->d_progs);
  if (s->h_progs) cudaFreeHost(s->h_progs);
  if (s->d_counts) cudaFree(s->d_counts);
  for (int b = 0; b < 2; b++) {
    if (s->h_witems_buf[b]) cudaFreeHost(s->h_witems_buf[b]);
    if (s->h_counts_buf[b]) cudaFreeHost(s->h_counts_buf[b]);
    if (s->d_items_buf[b]) cudaFree(s->d_items_buf[b]);
    if (s->h_items_buf[b]) cudaFreeHost(s->h_items_buf[b]);
  }
  if (s->d_slot_out) cudaFree(s->d_slot_out);
  if (s->h_slot_out) cudaFreeHost(s->h_slot_out);
  if (s->d_scan_total) cudaFree(s->d_scan_total);
  if (s->h_models) cudaFreeHost(s->h_models);
  for (auto& pair : s->evs)
    for (auto& ev : pair)
      if (ev) cudaEventDestroy(ev);
  if (s->uploaded) cudaEventDestroy(s->uploaded);
  if (s->upload) cudaStreamDestroy(s->upload);
  if (s->copies) cudaStreamDestroy(s->copies);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
