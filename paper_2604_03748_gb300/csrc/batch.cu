// Batched frames: many plumes of different grid and billboard sizes per call.
// Every stage is one launch over all plumes -- staging, the three passes of
// the segmented guide march, each network layer (grouped tensor-core
// convolutions and adapters), shading -- so the launch count does not grow
// with the number of plumes.  The per-plume tables the kernels read live in one
// device block that is refreshed from one pinned host block per call, which
// lets a captured CUDA graph pick up new cameras, lights and options on every
// replay.  An autotuner picks the segment length of the march, the march grid
// and the convolutions' CTAs per SM by timing candidates on the actual batch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nsl_internal.cuh"

using namespace nsl;

namespace {

struct Tables {                       // one pinned host block, mirrored on the device
  MarchPlume march[kMaxGroup];
  int tile_starts[kMaxGroup + 1];
  int item_starts[kMaxGroup + 1];
  int tile_counts[kMaxGroup];
  StageItem stage[kMaxGroup];
  int stage_starts[kMaxGroup + 1];
  ShadeArgs shade[kMaxGroup];
  int shade_starts[kMaxGroup + 1];
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Pinned host copies of the tables: a ring for ordinary renders (a slot is
// rewritten only after the copy that last read it has run) and one slot owned
// by the captured graph, whose copy node reads it at every replay.
constexpr int kRing = 3;
constexpr int kGraphSlot = kRing;

// Launch totals baked into a captured graph; a table update must keep them.
struct Totals {
  int n, tiles, items, sblocks, nshade, hblocks, precision;
  bool operator==(const Totals& o) const {
    return n == o.n && tiles == o.tiles && items == o.items && sblocks == o.sblocks &&
           nshade == o.nshade && hblocks == o.hblocks && precision == o.precision;
  }
};

}  // namespace

struct nsl_batch {
  int max_plumes = 0;
  std::vector<float> params;
  NetLayout layout{};
  NetF32Weights* wf = nullptr;
  NetTcWeights* wtc[kTcElems] = {};  // FP16, BF16, FP8, split BF16
  // device memory, grown on demand (never while a graph is being captured)
  void* staged = nullptr;  size_t staged_bytes = 0;
  void* seg = nullptr;     size_t seg_bytes = 0;
  void* net = nullptr;     size_t net_bytes = 0;
  Tables* host[kRing + 1] = {};    // pinned
  cudaEvent_t host_done[kRing] = {};
  int next_slot = 0;
  Tables* dev = nullptr;
  int* counter = nullptr;
  unsigned int* err_host = nullptr;
  unsigned int* err_dev = nullptr;
  // tuning
  int seg_len = kMarchSegLen;
  int seg_blocks_per_sm = 0;       // 0 = occupancy maximum
  int conv_ctas = 4;
  int tile_log2 = kMarchTXLog2;    // march tile: 2^tile_log2 x 2^(5 - tile_log2) pixels
  int persistent_march = 1;        // 1: the march as one cooperative launch, 0: three passes
  // captured graph
  cudaGraphExec_t exec = nullptr;
  bool capturing = false;
  Totals graph_totals{};
  std::vector<nsl_plume> graph_plumes;  // buffers and sizes of the capture
};

namespace {

void drop_graph(nsl_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_plumes.clear();
}

// Grow a device region; a captured graph that points into the old region is
// dropped (a later nsl_batch_launch_graph reports that there is none).
nsl_status grow(nsl_batch* b, void** p, size_t* have, size_t need, cudaStream_t s,
                const char* what) {
  if (need <= *have) return NSL_OK;
  if (b->capturing)
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch: %s would grow during graph capture or update", what);
  NSL_CUDA_TRY(cudaStreamSynchronize(s));
  drop_graph(b);
  cudaFree(*p);
  *p = nullptr;
  *have = 0;
  NSL_CUDA_TRY(cudaMalloc(p, need));
  *have = need;
  return NSL_OK;
}

nsl_status validate_plume(const nsl_plume& pl, int k, bool prestaged) {
  char fn[64];
  std::snprintf(fn, sizeof fn, "nsl_batch: plume %d", k);
  const nsl_grid_desc& g = pl.grid;
  if (!grid_dims_ok(g.nx, g.ny, g.nz) || (g.dtype != NSL_F32 && g.dtype != NSL_F16) || !(g.sigma_scale >= 0.f))
    return fail(NSL_ERR_INVALID_ARG, "%s: bad grid", fn);
  if ((!pl.density_dev && !prestaged) || !pl.guide_dev || !pl.lightmaps_dev)
    return fail(NSL_ERR_INVALID_ARG, "%s: NULL buffer", fn);
  const uintptr_t bits = reinterpret_cast<uintptr_t>(pl.density_dev) |
                         reinterpret_cast<uintptr_t>(pl.mask_dev) |
                         reinterpret_cast<uintptr_t>(pl.guide_dev) |
                         reinterpret_cast<uintptr_t>(pl.lightmaps_dev) |
                         reinterpret_cast<uintptr_t>(pl.rgba_dev);
  if (bits & 15u) return fail(NSL_ERR_INVALID_ARG, "%s: buffers must be 16-byte aligned", fn);
  return check_camera_basic(&pl.camera, fn);
}

}  // namespace

namespace nsl {
// Device scratch one plume takes in a batch: segment starts of the march and
// the network workspace (each rounded up to 256 bytes).
void batch_plume_scratch(const nsl_plume& p, int seg_len, size_t* seg_bytes, size_t* net_bytes, int precision) {
  const size_t P = (size_t)p.camera.width * p.camera.height;
  const int maxseg = march_max_segments(p.grid.nx, p.grid.ny, p.grid.nz, p.step_voxels, seg_len);
  *seg_bytes = align256(P * sizeof(int)) + align256(3 * (size_t)maxseg * P * sizeof(float));
  const int elem = tc_elem_of(precision);
  *net_bytes = align256(net_tc_workspace_bytes(p.camera.width, p.camera.height, elem < 0 ? 0 : elem));
}
}  // namespace nsl

namespace {

// Fill host table slot `T` for this batch and size every device region.
// Where prestaged[k] is set, plume k's grid is already staged there (padded
// quad layout) and is not staged again.
nsl_status prepare(nsl_batch* b, Tables& T, const nsl_plume* pl, int n, const nsl_march_opts* opts,
                   int precision, cudaStream_t s, std::vector<NetImage>* imgs,
                   std::vector<void*>* ws, Totals* tot, const float* const* prestaged) {
  if (n < 1 || n > b->max_plumes || n > kMaxGroup)
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch: n must be in [1, %d]", b->max_plumes);
  if (tc_elem_of(precision) < 0)
    return fail(NSL_ERR_UNSUPPORTED, "nsl_batch: batched network needs NSL_PREC_BF16, F16, FP8 or BF16X3");
  size_t staged = 0, seg = 0, net = 0;
  std::vector<size_t> off_staged(n), off_seg(n), off_net(n);
  std::vector<int> maxseg(n);
  for (int k = 0; k < n; ++k) {
    nsl_status st = validate_plume(pl[k], k, prestaged && prestaged[k]);
    if (st != NSL_OK) return st;
    const nsl_grid_desc& g = pl[k].grid;
    off_staged[k] = staged;
    if (!(prestaged && prestaged[k])) staged += align256(staged_grid_bytes(g));
    maxseg[k] = march_max_segments(g.nx, g.ny, g.nz, pl[k].step_voxels, b->seg_len);
    size_t sb, nb;
    batch_plume_scratch(pl[k], b->seg_len, &sb, &nb, precision);
    off_seg[k] = seg;
    seg += sb;
    off_net[k] = net;
    net += nb;
  }
  nsl_status st = grow(b, &b->staged, &b->staged_bytes, staged, s, "staged grids");
  if (st != NSL_OK) return st;
  if ((st = grow(b, &b->seg, &b->seg_bytes, seg, s, "march scratch")) != NSL_OK) return st;
  if ((st = grow(b, &b->net, &b->net_bytes, net, s, "network workspace")) != NSL_OK) return st;

  int tiles = 0, items = 0, sblocks = 0, hblocks = 0, nshade = 0;
  imgs->clear();
  ws->clear();
  for (int k = 0; k < n; ++k) {
    const nsl_plume& p = pl[k];
    MarchPlume& m = T.march[k];
    st = fill_march_plume(p.grid, p.camera, p.step_voxels, opts, "nsl_batch", &m);
    if (st != NSL_OK) return st;
    if (m.shadow_volume)
      return fail(NSL_ERR_UNSUPPORTED, "nsl_batch: shadow_volume is for the single-plume entry points");
    m.tx_log2 = b->tile_log2;
    m.tiles_x = (p.camera.width + (1 << b->tile_log2) - 1) >> b->tile_log2;
    const size_t P = (size_t)p.camera.width * p.camera.height;
    const bool pre = prestaged && prestaged[k];
    float* staged_k = pre ? const_cast<float*>(prestaged[k])
                          : reinterpret_cast<float*>(static_cast<char*>(b->staged) + off_staged[k]);
    m.vol = staged_k;
    m.staged_half = p.grid.dtype == NSL_F16 ? 1 : 0;   // float16 grids stay float16 quads
    m.scl = p.grid.sigma_scale;
    m.guide = p.guide_dev;
    m.seg_len = b->seg_len;
    char* sb = static_cast<char*>(b->seg) + off_seg[k];
    m.seg_nef = reinterpret_cast<int*>(sb);
    m.seg_tau = reinterpret_cast<float*>(sb + align256(P * sizeof(int)));
    m.seg_comp = m.seg_tau + (size_t)maxseg[k] * P;
    m.seg_L = m.seg_comp + (size_t)maxseg[k] * P;
    const int nt = march_tiles(p.camera.width, p.camera.height, b->tile_log2);
    T.tile_starts[k] = tiles;
    T.item_starts[k] = items;
    T.tile_counts[k] = nt;
    tiles += nt;
    items += nt * maxseg[k];
    StageItem& si = T.stage[k];
    si = StageItem{p.density_dev, p.mask_dev, staged_k, p.grid.nx, p.grid.ny, p.grid.nz,
                   p.grid.dtype, p.grid.sigma_scale, p.grid.dtype == NSL_F16 ? 1 : 0};
    T.stage_starts[k] = sblocks;
    if (!pre) sblocks += stage_batch_blocks(si);
    if (p.rgba_dev) {
      ShadeArgs& a = T.shade[nshade];
      a = ShadeArgs{};
      a.lm = p.lightmaps_dev;
      a.rgba = p.rgba_dev;
      a.W = p.camera.width;
      a.H = p.camera.height;
      st = shade_matrix(p.camera, &p.light, 1, a.M, "nsl_batch");
      if (st != NSL_OK) return st;
      T.shade_starts[nshade] = hblocks;
      hblocks += (int)((P / 4 + 255) / 256);
      ++nshade;
    }
    const double diag = std::sqrt((double)p.grid.nx * p.grid.nx + (double)p.grid.ny * p.grid.ny +
                                  (double)p.grid.nz * p.grid.nz);
    imgs->push_back(NetImage{p.guide_dev, p.lightmaps_dev, p.camera.height, p.camera.width,
                             (float)(1.0 / diag)});
    ws->push_back(static_cast<char*>(b->net) + off_net[k]);
  }
  T.tile_starts[n] = tiles;
  T.item_starts[n] = items;
  T.stage_starts[n] = sblocks;
  T.shade_starts[nshade] = hblocks;
  *tot = Totals{n, tiles, items, sblocks, nshade, hblocks, precision};
  return NSL_OK;
}

nsl_status render(nsl_batch* b, const nsl_plume* pl, int n, const nsl_march_opts* opts,
                  int precision, cudaStream_t s, const float* const* prestaged = nullptr) {
  if (*reinterpret_cast<volatile unsigned int*>(b->err_host) != 0) {
    const unsigned code = *b->err_host;
    *b->err_host = 0;
    // a barrier that gave up may have left its words behind: start them afresh
    NSL_CUDA_TRY(cudaStreamSynchronize(s));
    NSL_CUDA_TRY(cudaMemset(b->counter, 0, 256));
    return fail(NSL_ERR_TIMEOUT, "nsl_batch: an earlier launch timed out waiting (code 0x%x)", code);
  }
  // host slot: the graph's own while capturing, else the next ring slot once
  // the copy that last read it has run
  int slot = kGraphSlot;
  if (!b->capturing) {
    slot = b->next_slot;
    b->next_slot = (b->next_slot + 1) % kRing;
    NSL_CUDA_TRY(cudaEventSynchronize(b->host_done[slot]));
  }
  Tables& T = *b->host[slot];
  std::vector<NetImage> imgs;
  std::vector<void*> ws;
  Totals tot{};
  nsl_status st = prepare(b, T, pl, n, opts, precision, s, &imgs, &ws, &tot, prestaged);
  if (st != NSL_OK) return st;
  const int nshade = tot.nshade;
  NSL_CUDA_TRY(cudaMemcpyAsync(b->dev, &T, sizeof(Tables), cudaMemcpyHostToDevice, s));
  if (!b->capturing) NSL_CUDA_TRY(cudaEventRecord(b->host_done[slot], s));
  else b->graph_totals = tot;
  cudaError_t e = launch_stage_batch(b->dev->stage, b->dev->stage_starts, n, T.stage_starts[n], s);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_batch: staging");
  int per_sm = march_segment_blocks_max();
  if (b->seg_blocks_per_sm > 0 && b->seg_blocks_per_sm < per_sm) per_sm = b->seg_blocks_per_sm;
  if (b->persistent_march)
    e = launch_march_persistent_batch(b->dev->march, b->dev->tile_starts, b->dev->item_starts, b->dev->tile_counts,
                                      n, T.tile_starts[n], T.item_starts[n], per_sm * num_sms(),
                                      reinterpret_cast<unsigned*>(b->counter), b->err_dev, s);
  else
    e = launch_march_segmented_batch(b->dev->march, b->dev->tile_starts, b->dev->item_starts,
                                     b->dev->tile_counts, n, T.tile_starts[n], T.item_starts[n],
                                     per_sm * num_sms(), b->counter, s);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_batch: march");
  const int elem = tc_elem_of(precision);
  if (!b->wtc[elem]) {
    if (b->capturing) return fail(NSL_ERR_INVALID_ARG, "nsl_batch: weights not built before capture");
    b->wtc[elem] = net_tc_create(b->params.data(), b->layout, elem, &e);
    if (!b->wtc[elem]) return cuda_fail(e, "nsl_batch: tensor-core weights");
  }
  const int saved = net_tc_ctas_per_sm();
  net_tc_set_ctas_per_sm(b->conv_ctas);
  e = net_tc_forward_group(b->wtc[elem], b->wf, imgs.data(), ws.data(), n, b->err_dev, s);
  net_tc_set_ctas_per_sm(saved);
  if (e != cudaSuccess) return cuda_fail(e, "nsl_batch: network");
  if (nshade) {
    e = launch_shade_batch(b->dev->shade, b->dev->shade_starts, nshade, T.shade_starts[nshade], s);
    if (e != cudaSuccess) return cuda_fail(e, "nsl_batch: shading");
  }
  return NSL_OK;
}

}  // namespace

namespace nsl {
nsl_status batch_render_prestaged(nsl_batch* b, const nsl_plume* plumes, const float* const* staged,
                                  int n, const nsl_march_opts* opts, int precision, cudaStream_t s) {
  return render(b, plumes, n, opts, precision, s, staged);
}

// Allocate the march and network scratch up front so that batches that fit in
// it never reallocate (and never synchronise the device).
nsl_status batch_reserve(nsl_batch* b, size_t seg_bytes, size_t net_bytes, cudaStream_t s) {
  nsl_status st = grow(b, &b->seg, &b->seg_bytes, seg_bytes, s, "march scratch");
  if (st != NSL_OK) return st;
  return grow(b, &b->net, &b->net_bytes, net_bytes, s, "network workspace");
}

int batch_seg_len(const nsl_batch* b) { return b->seg_len; }
}  // namespace nsl

extern "C" {

nsl_status nsl_batch_create(const void* blob, size_t blob_bytes, int max_plumes, nsl_batch** out) {
  if (!out) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_create: out is NULL");
  *out = nullptr;
  if (!blob || blob_bytes < 20) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_create: bad blob");
  if (max_plumes < 1 || max_plumes > kMaxGroup)
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_create: max_plumes must be in [1, %d]", kMaxGroup);
  const unsigned char* bb = static_cast<const unsigned char*>(blob);
  uint32_t ver, c0, nf;
  if (std::memcmp(bb, "NSLW", 4) != 0) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_create: bad magic");
  std::memcpy(&ver, bb + 4, 4);
  std::memcpy(&c0, bb + 8, 4);
  std::memcpy(&nf, bb + 12, 4);
  if (ver != 1 || (size_t)nf * 4 + 20 != blob_bytes)
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_create: blob version or size mismatch");
  NetLayout L{};
  if (!build_net_layout((int)c0, &L) || L.c0 != kC0)
    return fail(NSL_ERR_UNSUPPORTED, "nsl_batch_create: C0=%u (batches run C0=16)", c0);
  if (L.total != nf) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_create: parameter count");
  uint32_t chk = 0, stored;
  for (uint32_t i = 0; i < nf; ++i) {
    uint32_t w;
    std::memcpy(&w, bb + 16 + 4 * (size_t)i, 4);
    chk += w;
  }
  std::memcpy(&stored, bb + 16 + 4 * (size_t)nf, 4);
  if (chk != stored) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_create: blob checksum mismatch");
  nsl_batch* b = new nsl_batch();
  b->max_plumes = max_plumes;
  b->layout = L;
  b->params.resize(nf);
  std::memcpy(b->params.data(), bb + 16, (size_t)nf * 4);
  cudaError_t e;
  b->wf = net_f32_create(b->params.data(), L, &e);
  if (!b->wf) { nsl_batch_destroy(b); return cuda_fail(e, "nsl_batch_create: weights"); }
  for (int i = 0; i <= kRing; ++i) {
    if ((e = cudaHostAlloc(reinterpret_cast<void**>(&b->host[i]), sizeof(Tables), cudaHostAllocDefault)) != cudaSuccess ||
        (i < kRing && (e = cudaEventCreateWithFlags(&b->host_done[i], cudaEventDisableTiming)) != cudaSuccess)) {
      nsl_batch_destroy(b);
      return cuda_fail(e, "nsl_batch_create: host tables");
    }
    std::memset(b->host[i], 0, sizeof(Tables));
  }
  if ((e = cudaMalloc(reinterpret_cast<void**>(&b->dev), sizeof(Tables))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void**>(&b->counter), 256)) != cudaSuccess ||
      (e = cudaMemset(b->counter, 0, 256)) != cudaSuccess ||
      (e = cudaHostAlloc(reinterpret_cast<void**>(&b->err_host), sizeof(unsigned int), cudaHostAllocMapped)) != cudaSuccess) {
    nsl_batch_destroy(b);
    return cuda_fail(e, "nsl_batch_create: allocation");
  }
  *b->err_host = 0;
  if ((e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&b->err_dev), b->err_host, 0)) != cudaSuccess) {
    nsl_batch_destroy(b);
    return cuda_fail(e, "nsl_batch_create: error word");
  }
  *out = b;
  return NSL_OK;
}

void nsl_batch_destroy(nsl_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  drop_graph(b);
  net_f32_destroy(b->wf);
  for (NetTcWeights* w : b->wtc) net_tc_destroy(w);
  cudaFree(b->staged);
  cudaFree(b->seg);
  cudaFree(b->net);
  cudaFree(b->dev);
  cudaFree(b->counter);
  for (int i = 0; i <= kRing; ++i) {
    if (b->host[i]) cudaFreeHost(b->host[i]);
    if (i < kRing && b->host_done[i]) cudaEventDestroy(b->host_done[i]);
  }
  if (b->err_host) cudaFreeHost(b->err_host);
  delete b;
}

nsl_status nsl_batch_render(nsl_batch* b, const nsl_plume* plumes, int n,
                            const nsl_march_opts* opts, int precision, void* stream) {
  if (!b || !plumes) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_render: NULL argument");
  return render(b, plumes, n, opts, precision, static_cast<cudaStream_t>(stream));
}

nsl_status nsl_batch_capture_graph(nsl_batch* b, const nsl_plume* plumes, int n,
                                   const nsl_march_opts* opts, int precision, void* stream) {
  if (!b || !plumes) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_capture_graph: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_capture_graph: needs a non-default stream");
  // one ordinary render first: every buffer, weight set and launch configuration
  // is created outside the capture
  nsl_status st = render(b, plumes, n, opts, precision, s);
  if (st != NSL_OK) return st;
  NSL_CUDA_TRY(cudaStreamSynchronize(s));
  drop_graph(b);
  NSL_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  b->capturing = true;
  st = render(b, plumes, n, opts, precision, s);
  b->capturing = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != NSL_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "nsl_batch_capture_graph: end capture");
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(e, "nsl_batch_capture_graph: instantiate");
  }
  b->graph_plumes.assign(plumes, plumes + n);
  return NSL_OK;
}

nsl_status nsl_batch_update_graph(nsl_batch* b, const nsl_plume* plumes, int n,
                                  const nsl_march_opts* opts) {
  if (!b || !plumes || !b->exec)
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_update_graph: no captured graph");
  if (n != (int)b->graph_plumes.size())
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_update_graph: the graph was captured for %d plumes",
                (int)b->graph_plumes.size());
  // the launches, kernel arguments and buffers baked into the graph must stay
  // valid: same buffers, grid and billboard sizes and step; cameras (pose,
  // projection), lights, sigma scales and march options may change
  for (int k = 0; k < n; ++k) {
    const nsl_plume &a = plumes[k], &c = b->graph_plumes[k];
    if (a.density_dev != c.density_dev || a.mask_dev != c.mask_dev || a.guide_dev != c.guide_dev ||
        a.lightmaps_dev != c.lightmaps_dev || a.rgba_dev != c.rgba_dev || a.grid.nx != c.grid.nx ||
        a.grid.ny != c.grid.ny || a.grid.nz != c.grid.nz || a.grid.dtype != c.grid.dtype ||
        a.camera.width != c.camera.width || a.camera.height != c.camera.height ||
        a.step_voxels != c.step_voxels)
      return fail(NSL_ERR_INVALID_ARG,
                  "nsl_batch_update_graph: plume %d changes a buffer, a size or the step of the capture", k);
  }
  std::vector<NetImage> imgs;
  std::vector<void*> ws;
  Totals tot{};
  Tables scratch;
  b->capturing = true;  // refuse any growth
  nsl_status st = prepare(b, scratch, plumes, n, opts, b->graph_totals.precision, nullptr, &imgs, &ws,
                          &tot, nullptr);
  b->capturing = false;
  if (st != NSL_OK) return st;
  if (!(tot == b->graph_totals))
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_update_graph: launch sizes differ from the capture");
  std::memcpy(b->host[kGraphSlot], &scratch, sizeof(Tables));
  return NSL_OK;
}

nsl_status nsl_batch_launch_graph(nsl_batch* b, void* stream) {
  if (!b || !b->exec) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_launch_graph: no captured graph");
  NSL_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return NSL_OK;
}

nsl_status nsl_batch_set_tuning(nsl_batch* b, int seg_len, int march_blocks_per_sm,
                                int conv_ctas_per_sm) {
  if (!b) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_set_tuning: NULL batch");
  if (seg_len < 1 || seg_len > 64 || march_blocks_per_sm < 0 || march_blocks_per_sm > 16 ||
      conv_ctas_per_sm < 1 || conv_ctas_per_sm > 4)
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_set_tuning: value out of range");
  // a captured graph holds the old segment layout and launch shapes
  if (seg_len != b->seg_len || march_blocks_per_sm != b->seg_blocks_per_sm ||
      conv_ctas_per_sm != b->conv_ctas) {
    cudaDeviceSynchronize();
    drop_graph(b);
  }
  b->seg_len = seg_len;
  b->seg_blocks_per_sm = march_blocks_per_sm;
  b->conv_ctas = conv_ctas_per_sm;
  return NSL_OK;
}

nsl_status nsl_batch_set_march_tile(nsl_batch* b, int tile_width) {
  if (!b) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_set_march_tile: NULL batch");
  const int lg = tile_width == 2 ? 1 : tile_width == 4 ? 2 : tile_width == 8 ? 3 : tile_width == 16 ? 4 : -1;
  if (lg < 0) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_set_march_tile: width must be 2, 4, 8 or 16");
  if (lg != b->tile_log2) {
    cudaDeviceSynchronize();
    drop_graph(b);   // a captured graph holds the old tile counts
  }
  b->tile_log2 = lg;
  return NSL_OK;
}

nsl_status nsl_batch_set_march_form(nsl_batch* b, int persistent) {
  if (!b || (persistent != 0 && persistent != 1))
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_set_march_form: NULL batch or form not 0 / 1");
  if (persistent != b->persistent_march) {
    cudaDeviceSynchronize();
    drop_graph(b);
  }
  b->persistent_march = persistent;
  return NSL_OK;
}

nsl_status nsl_batch_get_march_form(const nsl_batch* b, int* persistent) {
  if (!b || !persistent) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_get_march_form: NULL argument");
  *persistent = b->persistent_march;
  return NSL_OK;
}

nsl_status nsl_batch_get_march_tile(const nsl_batch* b, int* tile_width) {
  if (!b || !tile_width) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_get_march_tile: NULL argument");
  *tile_width = 1 << b->tile_log2;
  return NSL_OK;
}

nsl_status nsl_batch_get_tuning(const nsl_batch* b, int* seg_len, int* march_blocks_per_sm,
                                int* conv_ctas_per_sm) {
  if (!b || !seg_len || !march_blocks_per_sm || !conv_ctas_per_sm)
    return fail(NSL_ERR_INVALID_ARG, "nsl_batch_get_tuning: NULL argument");
  *seg_len = b->seg_len;
  *march_blocks_per_sm = b->seg_blocks_per_sm;
  *conv_ctas_per_sm = b->conv_ctas;
  return NSL_OK;
}

// Autotuner: time each candidate of the march (one persistent launch or three
// passes x tile shape x segment length x march blocks per SM), then of the
// convolutions' CTAs per SM, on this batch
// with CUDA events (median of 3 after one warm-up) and keep the fastest; with a
// cache path, a result recorded for the same batch signature is reused and new
// results are appended.
nsl_status nsl_batch_autotune(nsl_batch* b, const nsl_plume* plumes, int n,
                              const nsl_march_opts* opts, int precision, const char* cache_path,
                              void* stream, float* best_ms) {
  if (!b || !plumes) return fail(NSL_ERR_INVALID_ARG, "nsl_batch_autotune: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // batch signature: sizes, steps and precision
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) { h = (h ^ v) * 1099511628211ull; };
  mix((unsigned long long)n);
  mix((unsigned long long)precision);
  for (int k = 0; k < n; ++k) {
    mix((unsigned long long)plumes[k].grid.nx);
    mix((unsigned long long)plumes[k].grid.ny);
    mix((unsigned long long)plumes[k].grid.nz);
    mix((unsigned long long)plumes[k].camera.width);
    mix((unsigned long long)plumes[k].camera.height);
    unsigned int sb;
    std::memcpy(&sb, &plumes[k].step_voxels, 4);
    mix(sb);
  }
  char key[32];
  std::snprintf(key, sizeof key, "%016llx", h);
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[256];
      while (std::fgets(line, sizeof line, f)) {
        char k2[32];
        int a, c, d, tw, pf;
        float ms;
        if (std::sscanf(line, " {\"key\": \"%31[0-9a-f]\", \"seg_len\": %d, \"march_blocks_per_sm\": %d, "
                              "\"conv_ctas_per_sm\": %d, \"march_tile_width\": %d, \"persistent_march\": %d, "
                              "\"ms\": %f}", k2, &a, &c, &d, &tw, &pf, &ms) == 7 &&
            std::strcmp(k2, key) == 0) {
          std::fclose(f);
          if (best_ms) *best_ms = ms;
          nsl_status st = nsl_batch_set_march_tile(b, tw);
          if (st == NSL_OK) st = nsl_batch_set_march_form(b, pf);
          return st == NSL_OK ? nsl_batch_set_tuning(b, a, c, d) : st;
        }
      }
      std::fclose(f);
    }
  }
  const int seg_lens[] = {4, 6, 8};
  const int conv_ctas[] = {1, 2, 4};
  const int tiles[] = {8, 4};
  const int forms[] = {1, 0};
  const int occ = march_segment_blocks_max();
  std::vector<int> march_bps = {0};
  for (int v : {5, 6}) if (v < occ) march_bps.push_back(v);
  cudaEvent_t e0, e1;
  NSL_CUDA_TRY(cudaEventCreate(&e0));
  NSL_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int bs = b->seg_len, bm = b->seg_blocks_per_sm, bc = b->conv_ctas, bt = 1 << b->tile_log2,
      bf = b->persistent_march;
  nsl_status st = NSL_OK;
  // median of three timed renders after one warm-up
  auto time_it = [&](float* med) {
    float t[3] = {0.f, 0.f, 0.f};
    for (int r = 0; r < 4 && st == NSL_OK; ++r) {
      cudaEventRecord(e0, s);
      st = render(b, plumes, n, opts, precision, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      if (r > 0) cudaEventElapsedTime(&t[r - 1], e0, e1);
    }
    const float a = t[0], c = t[1], d = t[2];
    *med = a > c ? (c > d ? c : (a > d ? d : a)) : (a > d ? a : (c > d ? d : c));
  };
  // the march's knobs (tile shape, segment length, CTAs per SM) with the
  // network's at their current value, then the network's CTAs per SM: the two
  // stages do not interact
  for (int pf : forms)
    for (int tw : tiles)
      for (int sl : seg_lens)
        for (int mb : march_bps) {
          nsl_batch_set_march_form(b, pf);
          nsl_batch_set_march_tile(b, tw);
          nsl_batch_set_tuning(b, sl, mb, bc);
          float med;
          time_it(&med);
          if (st != NSL_OK) break;
          if (med < best) { best = med; bs = sl; bm = mb; bt = tw; bf = pf; }
        }
  nsl_batch_set_march_form(b, bf);
  nsl_batch_set_march_tile(b, bt);
  for (int cc : conv_ctas) {
    if (st != NSL_OK) break;
    nsl_batch_set_tuning(b, bs, bm, cc);
    float med;
    time_it(&med);
    if (st != NSL_OK) break;
    if (med < best) { best = med; bc = cc; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NSL_OK) return st;
  nsl_batch_set_tuning(b, bs, bm, bc);
  if (best_ms) *best_ms = best;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "{\"key\": \"%s\", \"seg_len\": %d, \"march_blocks_per_sm\": %d, "
                      "\"conv_ctas_per_sm\": %d, \"march_tile_width\": %d, \"persistent_march\": %d, "
                      "\"ms\": %.4f}\n", key, bs, bm, bc, bt, bf, best);
      std::fclose(f);
    }
  }
  return NSL_OK;
}

}  // extern "C"
