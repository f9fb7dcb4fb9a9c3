// Serving: frame requests over plumes kept resident on the device.
//
// A plume's staged grid (padded quad layout) and its guide / lightmap / RGBA
// state live in a stream-ordered memory pool while the plume is resident.  One
// scheduler thread owns every launch: it retires finished batches (event
// queries), then fills each free batch slot with the oldest queued requests
// that can run now (their plume idle, at most one request per plume, within
// the slot's scratch), admitting plumes under the HBM budget by evicting the
// least recently used idle ones, and launches the batch (uploads + staging of
// newly admitted plumes, then one batched render) on the slot's stream.
// Slots run concurrently, so arrivals join the next batch while others are on
// the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nsl_internal.cuh"

using namespace nsl;

namespace {

using Clock = std::chrono::steady_clock;
int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}
size_t align256(size_t v) { return (v + 255) / 256 * 256; }

constexpr int kStatePlanes = 3 + 8 + 4;  // guide, lightmaps, rgba

struct PlumeRec {
  nsl_grid_desc grid{};
  const void* dens_host = nullptr;
  const uint8_t* mask_host = nullptr;
  bool dens_reg = false, mask_reg = false;
  size_t dens_bytes = 0, mask_bytes = 0;
  float step = 0.f;
  int max_w = 0, max_h = 0;
  bool removed = false;
  size_t staged_bytes = 0, state_bytes = 0;
  // residency
  bool resident = false;
  float* staged = nullptr;
  float* state = nullptr;
  bool busy = false;          // a request of this plume is in a launched (or forming) batch
  int pending = 0;            // queued + running requests
  uint64_t last_use = 0;
  int last_w = 0, last_h = 0;
};

enum ReqState { kQueued, kRunning, kDone, kFailed };

struct Req {
  int plume = -1;
  nsl_camera cam{};
  nsl_light light{};
  float* lm_out = nullptr;
  float* rgba_out = nullptr;
  int64_t t_sub = 0, t_done = 0;
  ReqState st = kQueued;
  nsl_status err = NSL_OK;
  std::string msg;
};

struct Slot {
  cudaStream_t stream = nullptr;
  nsl_batch* batch = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<uint64_t> reqs;
  void* up_dens = nullptr;
  size_t up_dens_bytes = 0;
  void* up_mask = nullptr;
  size_t up_mask_bytes = 0;
};

}  // namespace

struct nsl_server {
  nsl_server_opts o{};
  int device = 0;
  size_t seg_cap = 0, net_cap = 0, slot_scratch = 0;
  int seg_len = kMarchSegLen;
  cudaMemPool_t pool = nullptr;
  std::vector<PlumeRec> plumes;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> queue;
  uint64_t next_id = 1;
  uint64_t use_clock = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  size_t resident_bytes = 0, upload_bytes = 0;
  // statistics
  uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_reqs = 0;
  uint64_t admissions = 0, evictions = 0;
  double pixels = 0.0;
  std::vector<float> lat_ms;
  int64_t first_sub = 0, last_done = 0;
};

namespace {

size_t used_bytes(const nsl_server* S) {
  return S->resident_bytes + S->upload_bytes + S->slots.size() * S->slot_scratch;
}

nsl_plume plume_of(const PlumeRec& p, const Req& r) {
  nsl_plume q{};
  q.density_dev = nullptr;  // prestaged
  q.mask_dev = nullptr;
  q.grid = p.grid;
  q.camera = r.cam;
  q.step_voxels = p.step;
  q.light = r.light;
  const size_t P = (size_t)p.max_w * p.max_h;
  q.guide_dev = p.state;
  q.lightmaps_dev = r.lm_out ? r.lm_out : p.state + 3 * P;
  q.rgba_dev = r.rgba_out ? r.rgba_out : p.state + 11 * P;
  return q;
}

void evict(nsl_server* S, int idx, cudaStream_t s) {
  PlumeRec& p = S->plumes[idx];
  cudaFreeAsync(p.staged, s);
  cudaFreeAsync(p.state, s);
  p.staged = nullptr;
  p.state = nullptr;
  p.resident = false;
  S->resident_bytes -= p.staged_bytes + p.state_bytes;
  ++S->evictions;
}

// Grow one of a slot's upload buffers (stream-ordered, so the previous
// contents are no longer needed once earlier work on the stream has run).
bool grow_upload(nsl_server* S, Slot& sl, void** buf, size_t* have, size_t need) {
  if (need <= *have) return true;
  if (*buf) cudaFreeAsync(*buf, sl.stream);
  S->upload_bytes -= *have;
  *buf = nullptr;
  *have = 0;
  if (cudaMallocFromPoolAsync(buf, need, S->pool, sl.stream) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return false;
  }
  *have = need;
  S->upload_bytes += need;
  return true;
}

// Make plume idx resident: evict LRU idle plumes until it fits, allocate its
// staged grid and state, upload its density (and mask) and stage it, all on
// the slot's stream.
bool admit(nsl_server* S, int idx, Slot& sl) {
  PlumeRec& p = S->plumes[idx];
  const size_t need = p.staged_bytes + p.state_bytes;
  const size_t up_extra = (p.dens_bytes > sl.up_dens_bytes ? p.dens_bytes - sl.up_dens_bytes : 0) +
                          (p.mask_bytes > sl.up_mask_bytes ? p.mask_bytes - sl.up_mask_bytes : 0);
  while (used_bytes(S) + need + up_extra > S->o.hbm_budget_bytes) {
    int victim = -1;
    for (int pass = 0; pass < 2 && victim < 0; ++pass)
      for (int k = 0; k < (int)S->plumes.size(); ++k) {
        const PlumeRec& v = S->plumes[k];
        if (!v.resident || v.busy || k == idx) continue;
        if (pass == 0 && v.pending > 0) continue;  // first choice: plumes nobody waits for
        if (victim < 0 || v.last_use < S->plumes[victim].last_use) victim = k;
      }
    if (victim < 0) return false;
    evict(S, victim, sl.stream);
  }
  if (!grow_upload(S, sl, &sl.up_dens, &sl.up_dens_bytes, p.dens_bytes)) return false;
  if (p.mask_host && !grow_upload(S, sl, &sl.up_mask, &sl.up_mask_bytes, p.mask_bytes)) return false;
  void *staged = nullptr, *state = nullptr;
  if (cudaMallocFromPoolAsync(&staged, p.staged_bytes, S->pool, sl.stream) != cudaSuccess ||
      cudaMallocFromPoolAsync(&state, p.state_bytes, S->pool, sl.stream) != cudaSuccess) {
    cudaGetLastError();
    if (staged) cudaFreeAsync(staged, sl.stream);
    return false;
  }
  if (cudaMemcpyAsync(sl.up_dens, p.dens_host, p.dens_bytes, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
      (p.mask_host && cudaMemcpyAsync(sl.up_mask, p.mask_host, p.mask_bytes, cudaMemcpyHostToDevice,
                                      sl.stream) != cudaSuccess) ||
      (p.grid.dtype == NSL_F16
           ? launch_stage_volume_half(static_cast<const __half*>(sl.up_dens),
                                      p.mask_host ? static_cast<const uint8_t*>(sl.up_mask) : nullptr, p.grid.nx,
                                      p.grid.ny, p.grid.nz, static_cast<__half*>(staged), sl.stream)
           : launch_stage_volume(sl.up_dens, p.grid.dtype,
                                 p.mask_host ? static_cast<const uint8_t*>(sl.up_mask) : nullptr, p.grid.nx,
                                 p.grid.ny, p.grid.nz, p.grid.sigma_scale, static_cast<float*>(staged),
                                 sl.stream)) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(staged, sl.stream);
    cudaFreeAsync(state, sl.stream);
    return false;
  }
  p.staged = static_cast<float*>(staged);
  p.state = static_cast<float*>(state);
  p.resident = true;
  S->resident_bytes += need;
  ++S->admissions;
  return true;
}

void fail_request(nsl_server* S, uint64_t id, nsl_status st, const std::string& msg) {
  Req& r = S->reqs[id];
  r.st = kFailed;
  r.err = st;
  r.msg = msg;
  PlumeRec& p = S->plumes[r.plume];
  p.pending--;
  ++S->failed;
}

// Form and launch one batch on a free slot.  Returns true if anything changed.
bool launch_batch(nsl_server* S, Slot& sl) {
  std::vector<uint64_t> pick;
  std::vector<int> picked;
  std::vector<char> taken(S->queue.size(), 0);
  size_t seg = 0, net = 0, pix = 0;
  // two scans of the queue in arrival order: the first takes only small
  // requests (at most small_first_pixels), the second the rest; a plume
  // whose oldest queued request is passed over in a scan takes no later one
  // in that scan, which keeps every plume's requests in arrival order
  const int scans = S->o.small_first_pixels ? 2 : 1;
  for (int scan = 0; scan < scans; ++scan) {
    const bool small_only = scans == 2 && scan == 0;
    size_t qi = 0;
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it, ++qi) {
      if ((int)pick.size() >= S->o.max_batch) break;
      if (taken[qi]) continue;
      const uint64_t id = *it;
      Req& r = S->reqs[id];
      PlumeRec& p = S->plumes[r.plume];
      if (p.busy) continue;  // running elsewhere, already in this batch or held back: keeps per-plume order
      const size_t rpix = (size_t)r.cam.width * r.cam.height;
      if (small_only && rpix > S->o.small_first_pixels) {
        p.busy = true;       // its later requests wait for this one
        picked.push_back(-1 - r.plume);
        continue;
      }
      size_t sb, nb;
      const nsl_plume q = plume_of(p, r);
      batch_plume_scratch(q, S->seg_len, &sb, &nb, S->o.precision);
      if (seg + sb > S->seg_cap || net + nb > S->net_cap ||
          (!pick.empty() && S->o.max_batch_pixels && pix + rpix > S->o.max_batch_pixels)) {
        p.busy = true;  // keep later requests of this plume behind this one
        picked.push_back(-1 - r.plume);
        continue;
      }
      if (!p.resident && !admit(S, r.plume, sl)) {
        p.busy = true;
        picked.push_back(-1 - r.plume);
        continue;
      }
      p.busy = true;
      picked.push_back(r.plume);
      pick.push_back(id);
      taken[qi] = 1;
      seg += sb;
      net += nb;
      pix += rpix;
    }
    // plumes only held back during this scan become free again
    for (int& v : picked)
      if (v < 0) {
        S->plumes[-1 - v].busy = false;
        v = INT32_MAX;
      }
  }
  if (pick.empty()) return false;

  std::vector<nsl_plume> pl;
  std::vector<const float*> staged;
  for (uint64_t id : pick) {
    Req& r = S->reqs[id];
    PlumeRec& p = S->plumes[r.plume];
    pl.push_back(plume_of(p, r));
    staged.push_back(p.staged);
  }
  nsl_status st = batch_render_prestaged(sl.batch, pl.data(), staged.data(), (int)pl.size(), &S->o.march,
                                         S->o.precision, sl.stream);
  cudaError_t e = cudaSuccess;
  if (st == NSL_OK) e = cudaEventRecord(sl.done, sl.stream);
  std::unordered_map<uint64_t, bool> in_batch;
  for (uint64_t id : pick) in_batch[id] = true;
  std::deque<uint64_t> rest;
  for (uint64_t id : S->queue)
    if (!in_batch.count(id)) rest.push_back(id);
  S->queue.swap(rest);
  if (st != NSL_OK || e != cudaSuccess) {
    const std::string msg = st != NSL_OK ? std::string(nsl_last_error()) : std::string(cudaGetErrorString(e));
    for (uint64_t id : pick) {
      S->plumes[S->reqs[id].plume].busy = false;
      fail_request(S, id, st != NSL_OK ? st : NSL_ERR_CUDA, msg);
    }
    S->cv_done.notify_all();
    return true;
  }
  for (uint64_t id : pick) {
    Req& r = S->reqs[id];
    r.st = kRunning;
    PlumeRec& p = S->plumes[r.plume];
    p.last_use = ++S->use_clock;
    p.last_w = r.cam.width;
    p.last_h = r.cam.height;
  }
  sl.reqs = pick;
  sl.busy = true;
  ++S->batches;
  S->batched_reqs += pick.size();
  return true;
}

bool retire(nsl_server* S, Slot& sl) {
  const cudaError_t q = cudaEventQuery(sl.done);
  if (q == cudaErrorNotReady) return false;
  const int64_t t = now_ns();
  const std::string msg = q == cudaSuccess ? std::string() : std::string(cudaGetErrorString(q));
  for (uint64_t id : sl.reqs) {
    Req& r = S->reqs[id];
    PlumeRec& p = S->plumes[r.plume];
    p.busy = false;
    if (q == cudaSuccess) {
      r.st = kDone;
      r.t_done = t;
      p.pending--;
      ++S->completed;
      S->pixels += (double)r.cam.width * r.cam.height;
      S->lat_ms.push_back((float)((t - r.t_sub) * 1e-6));
      S->last_done = t;
    } else {
      fail_request(S, id, NSL_ERR_CUDA, msg);
    }
  }
  sl.reqs.clear();
  sl.busy = false;
  return true;
}

void worker_main(nsl_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  int idle_polls = 0;
  for (;;) {
    bool progress = false;
    for (Slot& sl : S->slots)
      if (sl.busy && retire(S, sl)) progress = true;
    if (progress) S->cv_done.notify_all();
    for (Slot& sl : S->slots)
      if (!sl.busy && !S->queue.empty() && launch_batch(S, sl)) progress = true;
    bool any_busy = false;
    for (const Slot& sl : S->slots) any_busy |= sl.busy;
    if (S->stop && S->queue.empty() && !any_busy) break;
    if (progress) {
      idle_polls = 0;
      continue;
    }
    if (any_busy) {
      // poll the slots' events: yield for a few rounds, then short sleeps
      lk.unlock();
      if (++idle_polls < 64) std::this_thread::yield();
      else std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else if (!S->queue.empty()) {
      // nothing runs and nothing could be launched: the queued requests can
      // never be admitted (cannot happen for plumes that passed the checks at
      // registration, kept as a guard against waiting forever)
      for (uint64_t id : S->queue)
        fail_request(S, id, NSL_ERR_BUDGET, "nsl_server: request cannot be admitted within the budget");
      S->queue.clear();
      S->cv_done.notify_all();
    } else {
      idle_polls = 0;
      S->cv_work.wait(lk);
    }
  }
}

nsl_status check_grid(const nsl_grid_desc* g) {
  if (!g || !grid_dims_ok(g->nx, g->ny, g->nz) || (g->dtype != NSL_F32 && g->dtype != NSL_F16) || !(g->sigma_scale >= 0.f))
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_add_plume: bad grid description");
  return NSL_OK;
}

void register_host(const void* p, size_t bytes, bool* reg) {
  *reg = false;
  if (!p || !bytes) return;
  const cudaError_t e = cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterDefault);
  if (e == cudaSuccess) *reg = true;
  else cudaGetLastError();  // already page-locked, or not registrable: copies still work
}

}  // namespace

extern "C" {

void nsl_default_server_opts(nsl_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hbm_budget_bytes = size_t(40) << 30;
  o->scratch_bytes_per_stream = 0;
  o->streams = 2;
  o->max_batch = 64;
  o->max_batch_pixels = size_t(1) << 20;
  o->small_first_pixels = size_t(256) * 256;
  o->precision = NSL_PREC_F16;
  nsl_default_march_opts(&o->march);
}

nsl_status nsl_server_create(const void* blob, size_t blob_bytes, const nsl_server_opts* opts,
                             nsl_server** out) {
  if (!out) return fail(NSL_ERR_INVALID_ARG, "nsl_server_create: out is NULL");
  *out = nullptr;
  nsl_server_opts o;
  nsl_default_server_opts(&o);
  if (opts) o = *opts;
  if (o.streams < 1 || o.streams > 4 || o.max_batch < 1 || o.max_batch > kMaxGroup ||
      tc_elem_of(o.precision) < 0)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_create: streams 1..4, max_batch 1..%d, precision F16/BF16/FP8/BF16X3",
                kMaxGroup);
  if (!o.scratch_bytes_per_stream) o.scratch_bytes_per_stream = o.hbm_budget_bytes / 8;
  if (o.scratch_bytes_per_stream * o.streams >= o.hbm_budget_bytes)
    return fail(NSL_ERR_BUDGET, "nsl_server_create: slot scratch (%zu x %d) leaves nothing of the budget",
                o.scratch_bytes_per_stream, o.streams);
  nsl_server* S = new nsl_server();
  S->o = o;
  S->slot_scratch = align256(o.scratch_bytes_per_stream / 2) * 2;
  S->seg_cap = S->net_cap = S->slot_scratch / 2;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(e, "nsl_server_create: device");
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->device;
  if ((e = cudaMemPoolCreate(&S->pool, &props)) != cudaSuccess) {
    delete S;
    return cuda_fail(e, "nsl_server_create: memory pool");
  }
  uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool for the next admission
  cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  S->slots.resize(o.streams);
  for (Slot& sl : S->slots) {
    nsl_status st = nsl_batch_create(blob, blob_bytes, o.max_batch, &sl.batch);
    // slots run concurrently: the march in three ordinary passes, since a
    // cooperative launch occupies every SM until all its CTAs fit at once
    if (st == NSL_OK) st = nsl_batch_set_march_form(sl.batch, 0);
    if (st == NSL_OK && ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
                         (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess))
      st = cuda_fail(e, "nsl_server_create: stream");
    if (st == NSL_OK) st = batch_reserve(sl.batch, S->seg_cap, S->net_cap, sl.stream);
    if (st != NSL_OK) {
      nsl_server_destroy(S);
      return st;
    }
  }
  S->seg_len = batch_seg_len(S->slots[0].batch);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return NSL_OK;
}

void nsl_server_destroy(nsl_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (uint64_t id : S->queue) fail_request(S, id, NSL_ERR_INVALID_ARG, "nsl_server: destroyed");
    S->queue.clear();
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  S->cv_done.notify_all();
  cudaStream_t s0 = S->slots.empty() ? nullptr : S->slots[0].stream;
  for (size_t k = 0; k < S->plumes.size(); ++k) {
    PlumeRec& p = S->plumes[k];
    if (p.resident) evict(S, (int)k, s0);
    if (p.dens_reg) cudaHostUnregister(const_cast<void*>(p.dens_host));
    if (p.mask_reg) cudaHostUnregister(const_cast<uint8_t*>(p.mask_host));
  }
  for (Slot& sl : S->slots) {
    if (sl.up_dens) cudaFreeAsync(sl.up_dens, s0 ? s0 : sl.stream);
    if (sl.up_mask) cudaFreeAsync(sl.up_mask, s0 ? s0 : sl.stream);
  }
  cudaDeviceSynchronize();
  for (Slot& sl : S->slots) {
    nsl_batch_destroy(sl.batch);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
}

nsl_status nsl_server_add_plume(nsl_server* S, const nsl_grid_desc* grid, const void* density_host,
                                const uint8_t* mask_host, float step, int max_w, int max_h,
                                int* plume_id) {
  if (!S || !density_host || !plume_id) return fail(NSL_ERR_INVALID_ARG, "nsl_server_add_plume: NULL argument");
  nsl_status st = check_grid(grid);
  if (st != NSL_OK) return st;
  if (!(step > 0.f) || max_w < 8 || max_h < 8 || max_w % 8 || max_h % 8 || max_w > 8192 || max_h > 8192)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_add_plume: step > 0, billboard multiples of 8 in [8, 8192]");
  PlumeRec p;
  p.grid = *grid;
  p.dens_host = density_host;
  p.mask_host = mask_host;
  const size_t cells = (size_t)grid->nx * grid->ny * grid->nz;
  p.dens_bytes = cells * (grid->dtype == NSL_F16 ? 2 : 4);
  p.mask_bytes = mask_host ? cells : 0;
  p.step = step;
  p.max_w = max_w;
  p.max_h = max_h;
  p.staged_bytes = align256(staged_grid_bytes(*grid));
  p.state_bytes = align256((size_t)kStatePlanes * max_w * max_h * sizeof(float));
  // the plume alone (with its upload buffers) next to the slots' scratch, and
  // a frame at its largest billboard inside one slot's scratch
  if (p.staged_bytes + p.state_bytes + p.dens_bytes + p.mask_bytes + S->slots.size() * S->slot_scratch >
      S->o.hbm_budget_bytes)
    return fail(NSL_ERR_BUDGET, "nsl_server_add_plume: the plume needs %zu bytes; the budget leaves %zu",
                p.staged_bytes + p.state_bytes + p.dens_bytes + p.mask_bytes,
                S->o.hbm_budget_bytes - S->slots.size() * S->slot_scratch);
  nsl_plume q{};
  q.grid = *grid;
  q.camera.width = max_w;
  q.camera.height = max_h;
  q.step_voxels = step;
  size_t sb, nb;
  batch_plume_scratch(q, S->seg_len, &sb, &nb, S->o.precision);
  if (sb > S->seg_cap || nb > S->net_cap)
    return fail(NSL_ERR_BUDGET, "nsl_server_add_plume: a %dx%d frame needs %zu + %zu bytes of scratch; a slot "
                "holds %zu + %zu", max_w, max_h, sb, nb, S->seg_cap, S->net_cap);
  register_host(density_host, p.dens_bytes, &p.dens_reg);
  register_host(mask_host, p.mask_bytes, &p.mask_reg);
  std::lock_guard<std::mutex> lk(S->mu);
  S->plumes.push_back(p);
  *plume_id = (int)S->plumes.size() - 1;
  return NSL_OK;
}

nsl_status nsl_server_remove_plume(nsl_server* S, int id) {
  if (!S) return fail(NSL_ERR_INVALID_ARG, "nsl_server_remove_plume: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (id < 0 || id >= (int)S->plumes.size() || S->plumes[id].removed)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_remove_plume: unknown plume %d", id);
  PlumeRec& p = S->plumes[id];
  if (p.pending > 0 || p.busy)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_remove_plume: plume %d has %d requests pending", id, p.pending);
  if (p.resident) {
    evict(S, id, S->slots[0].stream);
    --S->evictions;  // a removal is not an eviction
  }
  if (p.dens_reg) cudaHostUnregister(const_cast<void*>(p.dens_host));
  if (p.mask_reg) cudaHostUnregister(const_cast<uint8_t*>(p.mask_host));
  p.dens_reg = p.mask_reg = false;
  p.removed = true;
  return NSL_OK;
}

nsl_status nsl_server_submit(nsl_server* S, int id, const nsl_camera* cam, const nsl_light* light,
                             float* lm_out, float* rgba_out, uint64_t* request_id) {
  const int64_t t = now_ns();
  if (!S || !cam || !light || !request_id) return fail(NSL_ERR_INVALID_ARG, "nsl_server_submit: NULL argument");
  nsl_status st = check_camera_basic(cam, "nsl_server_submit");
  if (st != NSL_OK) return st;
  if ((reinterpret_cast<uintptr_t>(lm_out) | reinterpret_cast<uintptr_t>(rgba_out)) & 15u)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_submit: output buffers must be 16-byte aligned");
  std::lock_guard<std::mutex> lk(S->mu);
  if (id < 0 || id >= (int)S->plumes.size() || S->plumes[id].removed)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_submit: unknown plume %d", id);
  PlumeRec& p = S->plumes[id];
  if (cam->width > p.max_w || cam->height > p.max_h)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_submit: %dx%d exceeds the plume's %dx%d", cam->width,
                cam->height, p.max_w, p.max_h);
  Req r;
  r.plume = id;
  r.cam = *cam;
  r.light = *light;
  r.lm_out = lm_out;
  r.rgba_out = rgba_out;
  r.t_sub = t;
  const uint64_t rid = S->next_id++;
  S->reqs.emplace(rid, std::move(r));
  S->queue.push_back(rid);
  p.pending++;
  ++S->submitted;
  if (!S->first_sub) S->first_sub = t;
  *request_id = rid;
  S->cv_work.notify_one();
  return NSL_OK;
}

nsl_status nsl_server_wait(nsl_server* S, uint64_t rid, double timeout_ms, double* latency_ms) {
  if (!S) return fail(NSL_ERR_INVALID_ARG, "nsl_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(rid);
  if (it == S->reqs.end()) return fail(NSL_ERR_INVALID_ARG, "nsl_server_wait: unknown request %llu",
                                       (unsigned long long)rid);
  const auto until = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1e3));
  while (it->second.st == kQueued || it->second.st == kRunning) {
    if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
        (it->second.st == kQueued || it->second.st == kRunning))
      return fail(NSL_ERR_TIMEOUT, "nsl_server_wait: request %llu not done after %.1f ms",
                  (unsigned long long)rid, timeout_ms);
    it = S->reqs.find(rid);
  }
  const Req r = it->second;
  S->reqs.erase(it);
  if (r.st == kFailed) return fail(r.err, "%s", r.msg.c_str());
  if (latency_ms) *latency_ms = (r.t_done - r.t_sub) * 1e-6;
  return NSL_OK;
}

nsl_status nsl_server_drain(nsl_server* S, double timeout_ms) {
  if (!S) return fail(NSL_ERR_INVALID_ARG, "nsl_server_drain: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  const auto until = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1e3));
  auto idle = [&] {
    if (!S->queue.empty()) return false;
    for (const Slot& sl : S->slots)
      if (sl.busy) return false;
    return true;
  };
  while (!idle())
    if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && !idle())
      return fail(NSL_ERR_TIMEOUT, "nsl_server_drain: work still pending after %.1f ms", timeout_ms);
  // completed requests nobody waits for individually are dropped here
  for (auto it = S->reqs.begin(); it != S->reqs.end();)
    it = (it->second.st == kDone) ? S->reqs.erase(it) : std::next(it);
  return NSL_OK;
}

nsl_status nsl_server_plume_state(nsl_server* S, int id, const float** guide, const float** lm,
                                  const float** rgba, int* resident) {
  if (!S || !guide || !lm || !rgba || !resident)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_plume_state: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (id < 0 || id >= (int)S->plumes.size() || S->plumes[id].removed)
    return fail(NSL_ERR_INVALID_ARG, "nsl_server_plume_state: unknown plume %d", id);
  const PlumeRec& p = S->plumes[id];
  *resident = p.resident ? 1 : 0;
  const size_t P = (size_t)p.max_w * p.max_h;
  *guide = p.resident ? p.state : nullptr;
  *lm = p.resident ? p.state + 3 * P : nullptr;
  *rgba = p.resident ? p.state + 11 * P : nullptr;
  return NSL_OK;
}

nsl_status nsl_server_get_stats(nsl_server* S, nsl_server_stats* out) {
  if (!S || !out) return fail(NSL_ERR_INVALID_ARG, "nsl_server_get_stats: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = S->queue.size();
  for (const Slot& sl : S->slots) out->running += sl.reqs.size();
  out->batches = S->batches;
  out->admissions = S->admissions;
  out->evictions = S->evictions;
  out->pixels_completed = S->pixels;
  for (const PlumeRec& p : S->plumes) out->resident_plumes += p.resident ? 1 : 0;
  out->resident_bytes = S->resident_bytes;
  out->used_bytes = used_bytes(S);
  out->budget_bytes = S->o.hbm_budget_bytes;
  if (!S->lat_ms.empty()) {
    std::vector<float> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const size_t i = (size_t)std::min<double>((double)v.size() - 1, std::ceil(q * v.size()) - 1);
      return (double)v[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
  }
  out->mean_batch = S->batches ? (double)S->batched_reqs / S->batches : 0.0;
  out->busy_s = (S->last_done > S->first_sub && S->first_sub) ? (S->last_done - S->first_sub) * 1e-9 : 0.0;
  return NSL_OK;
}

nsl_status nsl_server_reset_stats(nsl_server* S) {
  if (!S) return fail(NSL_ERR_INVALID_ARG, "nsl_server_reset_stats: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  S->submitted = S->completed = S->failed = S->batches = S->batched_reqs = 0;
  S->admissions = S->evictions = 0;
  S->pixels = 0.0;
  S->lat_ms.clear();
  S->first_sub = S->last_done = 0;
  return NSL_OK;
}

}  // extern "C"
