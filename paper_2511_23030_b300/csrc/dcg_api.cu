// C ABI of the dcg library: context, chunk table, pinned host tier (stand-in
// for the paper's disk tier), device page pool with LRU eviction, and the
// render / loss calls (Sec. III-D, III-E).
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

namespace dcg {

struct Chunk {
  uint64_t key = 0;
  int32_t c[3] = {0, 0, 0};
  int64_t count = 0;
  std::vector<int32_t> host_pages;  // slots [p * page_g, (p+1) * page_g) of the chunk
  std::vector<int32_t> dev_pages;   // same layout on the device when resident
  bool resident = false;
  bool dirty = false;
  int64_t last_access = -1;
  uint64_t load_seq = 0;         // copy-stream sequence number of the last load
  cudaEvent_t ev_load = nullptr;  // recorded after the last load's copies
};

}  // namespace dcg

using namespace dcg;

struct dcg_render_state {
  dcg_ctx* ctx = nullptr;
  int64_t cap_pairs = 0, cap_inst = 0, cap_pix = 0, cap_tiles = 0, cap_n = 0;
  int V = 0;
  int64_t n = 0, n_pix = 0;
  int n_tiles = 0;
  bool valid = false;
  int gen = 0;
  dcg_gaussians g{};
  int tile_w = 16, tile_h = 16, stage = 128;
  int idx_bits = 1, view_bits = 0;
  DevCam* d_cams = nullptr;
  DevCam* h_cams = nullptr;
  cudaEvent_t ev_cams = nullptr;
  float4* rec = nullptr;
  float4* bin = nullptr;  // binning record per pair: 32 B (centre, conic, tile rectangle)
  float* depth = nullptr;
  uint32_t* touched = nullptr;
  short4* rect = nullptr;
  float4* grad2d = nullptr;
  u64 *list_a = nullptr, *list_b = nullptr, *inst_a = nullptr, *inst_b = nullptr;
  u64 *list_sorted = nullptr, *inst_sorted = nullptr;
  uint2* ranges = nullptr;
  float* T_final = nullptr;
  uint32_t* n_contrib = nullptr;
  DevCounters* counters = nullptr;
  u64* part = nullptr;
  uint32_t* hist = nullptr;
  int P = 592;
  std::vector<DevCam> cams_host;
};

struct dcg_ctx {
  dcg_config cfg{};
  int F = 0;   // parameter components per Gaussian
  int Fs = 0;  // stored components per Gaussian: F, or 3 F with the Adam moments (m then v)
  int device = 0;
  int num_sms = 148;
  std::string err;
  int tile_w = 16, tile_h = 16, stage = 128;
  cudaStream_t copy_stream = nullptr;
  cudaStream_t cull_stream = nullptr;  // dcg_cull_chunks without a mask: waits for nothing the caller queued
  cudaEvent_t ev_copy = nullptr, ev_compute = nullptr;
  unsigned* d_errword = nullptr;
  unsigned* h_errword = nullptr;
  // chunk table
  std::vector<Chunk> chunks;  // ascending key
  std::unordered_map<uint64_t, int32_t> index;
  int32_t* d_coords = nullptr;
  uint8_t* d_vis = nullptr;
  int32_t* d_list = nullptr;
  int32_t* d_nlist = nullptr;
  int32_t* h_list = nullptr;
  int32_t* h_nlist = nullptr;
  dcg_camera* d_cullcams = nullptr;
  dcg_camera* h_cullcams = nullptr;
  // page pools
  int64_t page_g = 2048, page_floats = 0;
  float* d_pool = nullptr;
  int64_t dev_pages = 0;
  std::vector<int32_t> dev_free;
  float* h_tier = nullptr;
  int64_t host_pages = 0;
  std::vector<int32_t> host_free;
  int64_t resident_g = 0;
  int64_t step = 0;
  uint64_t copy_seq = 0;
  // active buffer
  float* d_active = nullptr;
  int64_t n_active = 0;
  std::vector<uint64_t> active_keys;
  std::vector<int64_t> active_counts;  // the gathered chunks' counts at the gather
  bool active_valid = false;
  // The active buffer as a write-back copy of the listed chunks: active_fresh
  // means a scatter_back of the buffer itself made it the chunks' stored value
  // (a gather of the same list hands it out again), active_dirty that the copy
  // into the device pages is still deferred.
  bool active_fresh = false;
  bool active_dirty = false;
  // page descriptors (page, count, offset) in two slots used in turn, so that
  // filling one waits only for the upload of the gather before last; desc_slot
  // is the slot of the active set's descriptors (used by its write-back)
  long long* d_desc = nullptr;
  long long* h_desc = nullptr;
  int64_t max_desc = 0;
  int desc_slot = 0;
  cudaEvent_t ev_descs[2] = {nullptr, nullptr};
  int n_desc = 0;
  // staging for table updates
  uint64_t* d_keys = nullptr;
  int64_t keys_cap = 0;
  uint64_t* h_keys = nullptr;
  float* h_stage = nullptr;
  int64_t stage_cap = 0;
  // statistics
  int64_t loads = 0, evictions = 0, bytes_h2d = 0, bytes_d2h = 0;
  dcg_render_state* st0 = nullptr;
  DevCam* d_losscams = nullptr;
  DevCam* h_losscams = nullptr;
  float* d_losspart = nullptr;
  // SSIM term: 16 x 16 tile tables (host staging: [0, 16) for dcg_loss, [16, 32) for the window graph)
  DevCam* d_ssimcams = nullptr;
  DevCam* d_wssimcams = nullptr;
  DevCam* h_ssimcams = nullptr;
  float* d_ssimpart = nullptr;
  int64_t cap_ssim_tiles = 0;
  // loop closure: per-keyframe cull masks, chunk segments of the active set, keyframes
  uint8_t* d_lcmask = nullptr;
  long long* d_lcseg = nullptr;
  int* d_lcsegc = nullptr;
  LcView* d_lcview = nullptr;
  // LoG sampling: per-pixel flags, sample count
  uint32_t* d_lsflags = nullptr;
  u64* d_lscount = nullptr;
  u64* d_lsvcount = nullptr;  // samples per view of the last sampling call
  float* d_lctmp = nullptr;  // loop closure: permuted rows [Fs][n], the permutation,
  long long* d_lcperm = nullptr;  // the moved rows and their keys (later their destinations)
  long long* d_lcmidx = nullptr;
  u64* d_lcmkey = nullptr;
  int64_t lc_dev_cap = 0;
  u64* d_lcsegkey = nullptr;      // per gathered chunk: id, destination base (max_chunks each)
  long long* d_lcsegbase = nullptr;
  u64* d_lccnt = nullptr;         // transformed and moved row counts
  long long* d_amoff = nullptr;   // active map: first active row and table index per gathered chunk
  int32_t* d_amchunk = nullptr;
  uint8_t* d_vis_async = nullptr;  // union flags of dcg_cull_chunks_async (its own, so it may overlap a synchronous cull)
  long long* h_amoff = nullptr;   // their pinned staging, reused once ev_am shows the last upload consumed
  int32_t* h_amchunk = nullptr;
  cudaEvent_t ev_am = nullptr;
  cudaEvent_t ev_loss = nullptr;
  // injected faults (testing): the armed kind fires once, after fault_skip opportunities pass
  int fault_kind = DCG_FAULT_NONE;
  int fault_skip = 0;
  // load verification (config flag bit 2, or a short_copy fault armed): every chunk
  // load is checked against the checksum of its host pages before the gather returns
  bool verify_loads = false;
  unsigned long long* d_loadsum = nullptr;  // checksum of the arrived pages, one per pending check
  unsigned long long* h_loadsum = nullptr;  // pinned read-back
  std::vector<std::pair<uint64_t, unsigned long long>> load_checks;  // (chunk id, expected checksum)
  // captured window graph
  cudaStream_t cap_stream = nullptr;  // private stream for capture (the legacy stream cannot be captured)
  cudaGraphExec_t win_exec = nullptr;
  DevCam* h_wcams = nullptr;   // pinned camera staging read by the graph's copy node
  cudaEvent_t ev_win = nullptr;
  int win_V = 0;
  int win_W[kMaxViewsApi] = {}, win_H[kMaxViewsApi] = {};
  int win_launch[3] = {0, 0, 0};
  unsigned long long win_kernels = 0;
  // profiler
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next = 0;
  uint64_t ev_dropped = 0;  // marks not recorded since the last read (the pool was used up)
  cudaEvent_t open_ev[PH_COUNT] = {};
  struct Rec {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
};

namespace {

static_assert((int)PH_COUNT == (int)DCG_PH_COUNT && (int)PH_SAMPLE == (int)DCG_PH_SAMPLE &&
                  (int)PH_LOOP == (int)DCG_PH_LOOP && (int)PH_STALL == (int)DCG_PH_STALL,
              "phase numbering of the ABI and the library differ");

void prof_mark(void* h, int phase, bool begin, cudaStream_t s) {
  dcg_ctx* ctx = (dcg_ctx*)h;
  if (!ctx->prof_on) return;
  if (ctx->ev_next >= ctx->ev_pool.size()) {
    ctx->ev_dropped++;
    if (!begin) ctx->open_ev[phase] = nullptr;  // its interval is not recorded
    return;
  }
  cudaEvent_t e = ctx->ev_pool[ctx->ev_next++];
  cudaEventRecord(e, s);
  if (begin) {
    ctx->open_ev[phase] = e;
  } else if (ctx->open_ev[phase]) {
    ctx->recs.push_back({phase, ctx->open_ev[phase], e});
    ctx->open_ev[phase] = nullptr;
  }
}

ProfHook hook(dcg_ctx* ctx) {
  ProfHook p;
  if (ctx->prof_on) {
    p.h = ctx;
    p.mark = prof_mark;
  }
  return p;
}

dcg_status fail(dcg_ctx* ctx, dcg_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

#define CK(call)                                                                                         \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return fail(ctx, DCG_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

int nsh(int deg) { return (deg + 1) * (deg + 1); }

template <class T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
}

dcg_status upload_coords(dcg_ctx* ctx) {
  std::vector<int32_t> co(ctx->chunks.size() * 3);
  for (size_t k = 0; k < ctx->chunks.size(); ++k)
    for (int a = 0; a < 3; ++a) co[3 * k + a] = ctx->chunks[k].c[a];
  if (!co.empty()) CK(cudaMemcpy(ctx->d_coords, co.data(), co.size() * 4, cudaMemcpyHostToDevice));
  return DCG_OK;
}

float* host_page(dcg_ctx* ctx, int32_t p) { return ctx->h_tier + (int64_t)p * ctx->page_floats; }
float* dev_page(dcg_ctx* ctx, int32_t p) { return ctx->d_pool + (int64_t)p * ctx->page_floats; }

// Copy the used part (cnt slots of every component) of one page.
cudaError_t page_copy(dcg_ctx* ctx, float* dst, const float* src, int64_t cnt, cudaMemcpyKind kind, cudaStream_t s) {
  if (cnt <= 0) return cudaSuccess;
  const size_t pitch = (size_t)ctx->page_g * 4;
  if (cnt == ctx->page_g) return cudaMemcpyAsync(dst, src, (size_t)ctx->page_floats * 4, kind, s);
  return cudaMemcpy2DAsync(dst, pitch, src, pitch, (size_t)cnt * 4, (size_t)ctx->Fs, kind, s);
}

int64_t pages_for(dcg_ctx* ctx, int64_t count) { return (count + ctx->page_g - 1) / ctx->page_g; }

dcg_status evict_chunk(dcg_ctx* ctx, Chunk& ch) {
  if (!ch.resident) return DCG_OK;
  if (ctx->active_dirty && std::find(ctx->active_keys.begin(), ctx->active_keys.end(), ch.key) != ctx->active_keys.end())
    return fail(ctx, DCG_ERR_STATE, "eviction of an active chunk before its write-back");
  if (ch.dirty) {
    for (size_t p = 0; p < ch.dev_pages.size(); ++p) {
      const int64_t cnt = std::min<int64_t>(ctx->page_g, ch.count - (int64_t)p * ctx->page_g);
      CK(page_copy(ctx, host_page(ctx, ch.host_pages[p]), dev_page(ctx, ch.dev_pages[p]), cnt,
                   cudaMemcpyDeviceToHost, ctx->copy_stream));
      ctx->bytes_d2h += cnt * ctx->Fs * 4;
    }
    ch.dirty = false;
  }
  for (int32_t p : ch.dev_pages) ctx->dev_free.push_back(p);
  ch.dev_pages.clear();
  ch.resident = false;
  ctx->resident_g -= ch.count;
  ctx->evictions++;
  return DCG_OK;
}

// True (and disarmed) if the armed fault is `kind` and its skip count has run out.
bool fault_fires(dcg_ctx* ctx, int kind) {
  if (ctx->fault_kind != kind) return false;
  if (ctx->fault_skip > 0) {
    --ctx->fault_skip;
    return false;
  }
  ctx->fault_kind = DCG_FAULT_NONE;
  return true;
}

// Checksum of a chunk's host pages, the same definition as k_page_checksum:
// the sum over its used words w of w * (2 i + 1) mod 2^64, i the word's index
// in the chunk's page sequence ((page * Fs + component) * page_g + row).
unsigned long long host_checksum(const dcg_ctx* ctx, const Chunk& ch) {
  unsigned long long acc = 0ull;
  for (size_t p = 0; p < ch.host_pages.size(); ++p) {
    const int64_t cnt = std::min<int64_t>(ctx->page_g, ch.count - (int64_t)p * ctx->page_g);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(ctx->h_tier + (int64_t)ch.host_pages[p] * ctx->page_floats);
    for (int c = 0; c < ctx->Fs; ++c) {
      const unsigned long long base = ((unsigned long long)p * ctx->Fs + c) * (unsigned long long)ctx->page_g;
      for (int64_t j = 0; j < cnt; ++j)
        acc += (unsigned long long)src[(int64_t)c * ctx->page_g + j] * (2ull * (base + (unsigned long long)j) + 1ull);
    }
  }
  return acc;
}

dcg_status load_chunk(dcg_ctx* ctx, Chunk& ch) {
  const int64_t np = pages_for(ctx, ch.count);
  if ((int64_t)ctx->dev_free.size() < np) return fail(ctx, DCG_ERR_BUDGET, "device page pool exhausted");
  if (fault_fires(ctx, DCG_FAULT_H2D_FAIL)) return fail(ctx, DCG_ERR_FAULT, "injected host->device copy failure");
  const bool shorten = fault_fires(ctx, DCG_FAULT_SHORT_COPY);
  unsigned long long expect = 0ull;
  if (ctx->verify_loads) {
    // the host pages must be final: an eviction's device->host copy may still be running
    CK(cudaStreamSynchronize(ctx->copy_stream));
    expect = host_checksum(ctx, ch);
  }
  ch.dev_pages.resize((size_t)np);
  for (int64_t p = 0; p < np; ++p) {
    ch.dev_pages[(size_t)p] = ctx->dev_free.back();
    ctx->dev_free.pop_back();
    int64_t cnt = std::min<int64_t>(ctx->page_g, ch.count - p * ctx->page_g);
    float* dst = dev_page(ctx, ch.dev_pages[(size_t)p]);
    if (shorten && p == np - 1) {
      // injected short copy: the page's old contents are overwritten with a
      // pattern and only half of its rows are copied
      CK(cudaMemsetAsync(dst, 0xff, (size_t)ctx->page_floats * 4, ctx->copy_stream));
      cnt /= 2;
    }
    CK(page_copy(ctx, dst, host_page(ctx, ch.host_pages[(size_t)p]), cnt, cudaMemcpyHostToDevice, ctx->copy_stream));
    ctx->bytes_h2d += cnt * ctx->Fs * 4;
  }
  if (ctx->verify_loads) {
    const size_t slot = ctx->load_checks.size();
    if ((int64_t)slot >= ctx->cfg.max_chunks) return fail(ctx, DCG_ERR_CAPACITY, "too many unchecked loads");
    CK(cudaMemsetAsync(ctx->d_loadsum + slot, 0, sizeof(unsigned long long), ctx->copy_stream));
    for (int64_t p = 0; p < np; ++p) {
      const int64_t cnt = std::min<int64_t>(ctx->page_g, ch.count - p * ctx->page_g);
      launch_page_checksum(dev_page(ctx, ch.dev_pages[(size_t)p]), p, ctx->page_g, ctx->Fs, cnt,
                           ctx->d_loadsum + slot, ctx->copy_stream);
    }
    CK(cudaGetLastError());
    ctx->load_checks.push_back({ch.key, expect});
  }
  if (!ch.ev_load) CK(cudaEventCreateWithFlags(&ch.ev_load, cudaEventDisableTiming));
  CK(cudaEventRecord(ch.ev_load, ctx->copy_stream));
  ch.load_seq = ++ctx->copy_seq;
  ch.resident = true;
  ch.dirty = false;
  ctx->resident_g += ch.count;
  ctx->loads++;
  return DCG_OK;
}

dcg_status state_alloc(dcg_ctx* ctx, dcg_render_state* st) {
  const dcg_config& c = ctx->cfg;
  st->ctx = ctx;
  st->cap_n = c.max_active;
  st->cap_pairs = (int64_t)c.max_views * c.max_active;
  st->cap_inst = c.max_instances;
  st->cap_pix = c.max_pixels;
  st->cap_tiles = c.max_pixels / 16 + 64 * (int64_t)c.max_views + 64;  // generous bound incl. ragged edges
  st->P = ctx->num_sms * 8;  // partitions of the scans and sorts: 8 per SM keep enough loads in flight
  CK(dmalloc(&st->d_cams, kMaxViewsApi));
  CK(cudaHostAlloc((void**)&st->h_cams, sizeof(DevCam) * kMaxViewsApi, cudaHostAllocDefault));
  CK(cudaEventCreateWithFlags(&st->ev_cams, cudaEventDisableTiming));
  CK(dmalloc(&st->rec, 3 * (size_t)st->cap_pairs));
  CK(dmalloc(&st->depth, (size_t)st->cap_pairs));
  CK(dmalloc(&st->touched, (size_t)st->cap_pairs));
  CK(dmalloc(&st->rect, (size_t)st->cap_pairs));
  CK(dmalloc(&st->bin, 2 * (size_t)st->cap_pairs));
  CK(dmalloc(&st->grad2d, 3 * (size_t)st->cap_pairs));
  // the 2D gradient slots are zero between backward passes: the blends add
  // into them and the preprocess backward zeroes each slot it consumes
  CK(cudaMemset(st->grad2d, 0, sizeof(float4) * 3 * (size_t)st->cap_pairs));
  CK(dmalloc(&st->list_a, (size_t)st->cap_pairs));
  CK(dmalloc(&st->list_b, (size_t)st->cap_pairs));
  CK(dmalloc(&st->inst_a, (size_t)st->cap_inst));
  CK(dmalloc(&st->inst_b, (size_t)st->cap_inst));
  CK(dmalloc(&st->ranges, (size_t)st->cap_tiles));
  CK(dmalloc(&st->T_final, (size_t)st->cap_pix));
  CK(dmalloc(&st->n_contrib, (size_t)st->cap_pix));
  CK(dmalloc(&st->counters, 1));
  CK(dmalloc(&st->part, (size_t)st->P + 1));
  CK(dmalloc(&st->hist, 256 * ((size_t)st->P + 1)));
  return DCG_OK;
}

void state_free(dcg_render_state* st) {
  cudaFree(st->d_cams);
  if (st->h_cams) cudaFreeHost(st->h_cams);
  if (st->ev_cams) cudaEventDestroy(st->ev_cams);
  cudaFree(st->rec); cudaFree(st->depth); cudaFree(st->touched); cudaFree(st->rect); cudaFree(st->grad2d);
  cudaFree(st->bin);
  cudaFree(st->list_a); cudaFree(st->list_b); cudaFree(st->inst_a); cudaFree(st->inst_b);
  cudaFree(st->ranges); cudaFree(st->T_final); cudaFree(st->n_contrib); cudaFree(st->counters);
  cudaFree(st->part); cudaFree(st->hist);
}

bool valid_tile(int tw, int th) { return (tw == 16 && th == 16) || (tw == 32 && th == 16) || (tw == 32 && th == 32); }
// instance keys hold the global tile id in 20 bits (and the pair index in 28)
constexpr int kMaxTiles = 1 << 20;

bool valid_stage(int s) { return s == 16 || s == 32 || s == 64 || s == 96 || s == 128 || s == 192 || s == 256; }

dcg_status check_cams(dcg_ctx* ctx, const dcg_camera* cams, int V) {
  if (!cams || V <= 0 || V > ctx->cfg.max_views || V > kMaxViewsApi) return fail(ctx, DCG_ERR_ARG, "bad views");
  for (int v = 0; v < V; ++v) {
    const dcg_camera& c = cams[v];
    if (c.W <= 0 || c.H <= 0 || !(c.fx > 0) || !(c.fy > 0) || !(c.znear > 0) || !(c.zfar > c.znear))
      return fail(ctx, DCG_ERR_ARG, "bad camera");
  }
  return DCG_OK;
}

}  // namespace

extern "C" {

// Copies a deferred scatter_back of the active buffer into the device pages
// (on stream s, before anything reads, evicts or rewrites those pages).
// Device descriptors of the active set (the slot its gather filled).
const long long* active_desc(const dcg_ctx* ctx) { return ctx->d_desc + (size_t)ctx->desc_slot * 3 * ctx->max_desc; }

// The host staging of the other descriptor slot, once the upload that last
// used it has run; desc_upload() then sends nd descriptors and makes it current.
dcg_status desc_stage(dcg_ctx* ctx, long long** h) {
  const int slot = ctx->desc_slot ^ 1;
  CK(cudaEventSynchronize(ctx->ev_descs[slot]));
  *h = ctx->h_desc + (size_t)slot * 3 * ctx->max_desc;
  return DCG_OK;
}
dcg_status desc_upload(dcg_ctx* ctx, int nd, cudaStream_t s) {
  const int slot = ctx->desc_slot ^ 1;
  const size_t o = (size_t)slot * 3 * ctx->max_desc;
  if (nd > 0) CK(cudaMemcpyAsync(ctx->d_desc + o, ctx->h_desc + o, sizeof(long long) * 3 * nd, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(ctx->ev_descs[slot], s));
  ctx->desc_slot = slot;
  ctx->n_desc = nd;
  return DCG_OK;
}

dcg_status writeback_active(dcg_ctx* ctx, cudaStream_t s) {
  if (!ctx->active_dirty) return DCG_OK;
  ctx->active_dirty = false;
  if (!ctx->active_valid) return DCG_OK;
  launch_page_copy(false, ctx->d_pool, ctx->page_g, ctx->Fs, 0, ctx->Fs, active_desc(ctx), ctx->n_desc, ctx->d_active,
                   ctx->cfg.max_active, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->ev_compute, s));
  return DCG_OK;
}

void dcg_config_default(dcg_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->chunk_size = 4.0f;
  c->sh_degree = 3;
  c->device_budget = 6000000;
  c->host_capacity = 6000000;
  c->max_chunks = 8192;
  c->max_views = 8;
  c->max_active = 6000000;
  c->max_pixels = 8 * 1241 * 376;
  c->max_instances = 64 << 20;
  c->tile_w = 16;
  c->tile_h = 16;
  c->stage = 16;  // half-warp blends: the fastest launch on the benchmark window
  c->dfar = 100.0f;
  c->page_gaussians = 2048;
}

const char* dcg_last_error(const dcg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dcg_status dcg_create(const dcg_config* cfg, dcg_ctx** out) {
  if (!cfg || !out) return DCG_ERR_ARG;
  *out = nullptr;
  dcg_ctx* ctx = new dcg_ctx();
  ctx->cfg = *cfg;
  const dcg_config& c = ctx->cfg;
  dcg_status bad = DCG_OK;
  if (c.sh_degree < 0 || c.sh_degree > 3 || !(c.chunk_size > 0) || c.device_budget <= 0 || c.host_capacity <= 0 ||
      c.max_chunks <= 0 || c.max_views <= 0 || c.max_views > kMaxViewsApi || c.max_active <= 0 || c.max_pixels <= 0 ||
      c.max_instances <= 0 || c.max_instances >= (1ll << 32) || c.page_gaussians <= 0 ||
      (c.page_gaussians & (c.page_gaussians - 1)) != 0 || !valid_tile(c.tile_w, c.tile_h) || !valid_stage(c.stage) ||
      (int64_t)c.max_views * c.max_active > (1ll << 28) || (c.with_moments != 0 && c.with_moments != 1))
    bad = DCG_ERR_ARG;
  if (bad != DCG_OK) {
    delete ctx;
    return bad;
  }
  ctx->F = 11 + 3 * nsh(c.sh_degree);
  ctx->Fs = c.with_moments ? 3 * ctx->F : ctx->F;
  ctx->tile_w = c.tile_w;
  ctx->tile_h = c.tile_h;
  ctx->stage = c.stage;
  ctx->page_g = c.page_gaussians;
  ctx->page_floats = ctx->page_g * ctx->Fs;
  auto cleanup_fail = [&](dcg_status s) {
    dcg_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return cleanup_fail(DCG_ERR_CUDA);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return cleanup_fail(DCG_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&ctx->cull_stream, cudaStreamNonBlocking) != cudaSuccess) return cleanup_fail(DCG_ERR_CUDA);
  cudaEventCreateWithFlags(&ctx->ev_copy, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_compute, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_descs[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_descs[1], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_am, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_loss, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_win, cudaEventDisableTiming);
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return cleanup_fail(DCG_ERR_CUDA);
  if (cudaHostAlloc((void**)&ctx->h_wcams, sizeof(DevCam) * 2 * kMaxViewsApi, 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  if (dmalloc(&ctx->d_losspart, (size_t)loss_partials(ctx->num_sms)) != cudaSuccess ||
      dmalloc(&ctx->d_losscams, kMaxViewsApi) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_losscams, sizeof(DevCam) * kMaxViewsApi, 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  if (dmalloc(&ctx->d_lsflags, (size_t)c.max_pixels) != cudaSuccess || dmalloc(&ctx->d_lscount, 1) != cudaSuccess ||
      dmalloc(&ctx->d_lsvcount, kLsMaxViews) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  if (log_init() != cudaSuccess) return cleanup_fail(DCG_ERR_CUDA);
  ctx->cap_ssim_tiles = c.max_pixels / 16 + 64 * (int64_t)c.max_views + 64;
  if (dmalloc(&ctx->d_ssimcams, kMaxViewsApi) != cudaSuccess || dmalloc(&ctx->d_wssimcams, kMaxViewsApi) != cudaSuccess ||
      dmalloc(&ctx->d_ssimpart, 3 * (size_t)ctx->cap_ssim_tiles) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_ssimcams, sizeof(DevCam) * 2 * kMaxViewsApi, 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  if (ssim_init() != cudaSuccess) return cleanup_fail(DCG_ERR_CUDA);
  if (dmalloc(&ctx->d_lcmask, (size_t)kMaxViewsApi * c.max_chunks) != cudaSuccess ||
      dmalloc(&ctx->d_lcseg, (size_t)c.max_chunks) != cudaSuccess ||
      dmalloc(&ctx->d_lcsegc, (size_t)c.max_chunks) != cudaSuccess || dmalloc(&ctx->d_lcview, kMaxViewsApi) != cudaSuccess ||
      dmalloc(&ctx->d_lcsegkey, (size_t)c.max_chunks) != cudaSuccess ||
      dmalloc(&ctx->d_lcsegbase, (size_t)c.max_chunks) != cudaSuccess || dmalloc(&ctx->d_lccnt, 2) != cudaSuccess ||
      dmalloc(&ctx->d_amoff, (size_t)c.max_chunks) != cudaSuccess ||
      dmalloc(&ctx->d_amchunk, (size_t)c.max_chunks) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_amoff, sizeof(long long) * (size_t)c.max_chunks, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_amchunk, sizeof(int32_t) * (size_t)c.max_chunks, 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  if (dmalloc(&ctx->d_loadsum, (size_t)c.max_chunks) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_loadsum, sizeof(unsigned long long) * (size_t)c.max_chunks, 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  ctx->verify_loads = (c.flags & 4) != 0;
  if (const char* spec = std::getenv("DCG_FAULT")) {
    int32_t kind = 0, skip = 0;
    if (dcg_fault_parse(spec, &kind, &skip) != DCG_OK) return cleanup_fail(DCG_ERR_ARG);
    dcg_inject_fault(ctx, kind, skip);
  }
  if (dmalloc(&ctx->d_errword, 1) != cudaSuccess) return cleanup_fail(DCG_ERR_OOM);
  cudaMemset(ctx->d_errword, 0, sizeof(unsigned));
  if (cudaHostAlloc((void**)&ctx->h_errword, sizeof(unsigned), 0) != cudaSuccess) return cleanup_fail(DCG_ERR_OOM);
  // chunk table mirror
  if (dmalloc(&ctx->d_coords, 3 * (size_t)c.max_chunks) != cudaSuccess ||
      dmalloc(&ctx->d_vis, (size_t)c.max_chunks) != cudaSuccess || dmalloc(&ctx->d_list, (size_t)c.max_chunks) != cudaSuccess ||
      dmalloc(&ctx->d_vis_async, (size_t)c.max_chunks) != cudaSuccess ||
      dmalloc(&ctx->d_nlist, 1) != cudaSuccess || dmalloc(&ctx->d_cullcams, kMaxViewsApi) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  if (cudaHostAlloc((void**)&ctx->h_list, sizeof(int32_t) * c.max_chunks, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_nlist, sizeof(int32_t), 0) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_cullcams, sizeof(dcg_camera) * kMaxViewsApi, 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  // page pools: the budget in Gaussians plus one partly filled page per chunk that can be resident
  ctx->dev_pages = (c.device_budget + ctx->page_g - 1) / ctx->page_g + std::min<int64_t>(c.max_chunks, 4096);
  ctx->host_pages = (c.host_capacity + ctx->page_g - 1) / ctx->page_g + c.max_chunks;
  if (dmalloc(&ctx->d_pool, (size_t)(ctx->dev_pages * ctx->page_floats)) != cudaSuccess) return cleanup_fail(DCG_ERR_OOM);
  if (cudaHostAlloc((void**)&ctx->h_tier, sizeof(float) * (size_t)(ctx->host_pages * ctx->page_floats), 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  for (int64_t p = ctx->dev_pages - 1; p >= 0; --p) ctx->dev_free.push_back((int32_t)p);
  for (int64_t p = ctx->host_pages - 1; p >= 0; --p) ctx->host_free.push_back((int32_t)p);
  // active buffer and page descriptors
  if (dmalloc(&ctx->d_active, (size_t)ctx->Fs * c.max_active) != cudaSuccess) return cleanup_fail(DCG_ERR_OOM);
  ctx->max_desc = ctx->dev_pages;
  if (dmalloc(&ctx->d_desc, 2 * 3 * (size_t)ctx->max_desc) != cudaSuccess ||
      cudaHostAlloc((void**)&ctx->h_desc, sizeof(long long) * 2 * 3 * (size_t)ctx->max_desc, 0) != cudaSuccess)
    return cleanup_fail(DCG_ERR_OOM);
  ctx->st0 = new dcg_render_state();
  if (state_alloc(ctx, ctx->st0) != DCG_OK) return cleanup_fail(DCG_ERR_OOM);
  if (cudaDeviceSynchronize() != cudaSuccess) return cleanup_fail(DCG_ERR_CUDA);
  *out = ctx;
  return DCG_OK;
}

dcg_status dcg_destroy(dcg_ctx* ctx) {
  if (!ctx) return DCG_ERR_ARG;
  cudaDeviceSynchronize();
  if (ctx->st0) {
    state_free(ctx->st0);
    delete ctx->st0;
  }
  for (auto& ch : ctx->chunks)
    if (ch.ev_load) cudaEventDestroy(ch.ev_load);
  cudaFree(ctx->d_errword);
  if (ctx->h_errword) cudaFreeHost(ctx->h_errword);
  cudaFree(ctx->d_coords); cudaFree(ctx->d_vis); cudaFree(ctx->d_list); cudaFree(ctx->d_nlist); cudaFree(ctx->d_cullcams);
  cudaFree(ctx->d_vis_async);
  if (ctx->h_list) cudaFreeHost(ctx->h_list);
  if (ctx->h_nlist) cudaFreeHost(ctx->h_nlist);
  if (ctx->h_cullcams) cudaFreeHost(ctx->h_cullcams);
  cudaFree(ctx->d_pool);
  if (ctx->h_tier) cudaFreeHost(ctx->h_tier);
  cudaFree(ctx->d_active);
  cudaFree(ctx->d_desc);
  if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
  cudaFree(ctx->d_keys);
  if (ctx->h_keys) cudaFreeHost(ctx->h_keys);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->cull_stream) cudaStreamDestroy(ctx->cull_stream);
  if (ctx->ev_copy) cudaEventDestroy(ctx->ev_copy);
  if (ctx->ev_compute) cudaEventDestroy(ctx->ev_compute);
  for (cudaEvent_t e : ctx->ev_descs)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_loss) cudaEventDestroy(ctx->ev_loss);
  if (ctx->win_exec) cudaGraphExecDestroy(ctx->win_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->h_wcams) cudaFreeHost(ctx->h_wcams);
  cudaFree(ctx->d_lctmp);
  cudaFree(ctx->d_lcperm);
  cudaFree(ctx->d_lcmidx);
  cudaFree(ctx->d_lcmkey);
  cudaFree(ctx->d_lcsegkey);
  cudaFree(ctx->d_lcsegbase);
  cudaFree(ctx->d_lccnt);
  cudaFree(ctx->d_loadsum);
  if (ctx->h_loadsum) cudaFreeHost(ctx->h_loadsum);
  cudaFree(ctx->d_amoff);
  cudaFree(ctx->d_amchunk);
  if (ctx->h_amoff) cudaFreeHost(ctx->h_amoff);
  if (ctx->h_amchunk) cudaFreeHost(ctx->h_amchunk);
  if (ctx->ev_am) cudaEventDestroy(ctx->ev_am);
  if (ctx->ev_win) cudaEventDestroy(ctx->ev_win);
  for (auto& e : ctx->ev_pool) cudaEventDestroy(e);
  cudaFree(ctx->d_losscams);
  cudaFree(ctx->d_losspart);
  if (ctx->h_losscams) cudaFreeHost(ctx->h_losscams);
  cudaFree(ctx->d_lsflags);
  cudaFree(ctx->d_lscount);
  cudaFree(ctx->d_lsvcount);
  cudaFree(ctx->d_lcmask);
  cudaFree(ctx->d_lcseg);
  cudaFree(ctx->d_lcsegc);
  cudaFree(ctx->d_lcview);
  cudaFree(ctx->d_ssimcams);
  cudaFree(ctx->d_wssimcams);
  cudaFree(ctx->d_ssimpart);
  if (ctx->h_ssimcams) cudaFreeHost(ctx->h_ssimcams);
  delete ctx;
  return DCG_OK;
}

dcg_status dcg_fault_parse(const char* spec, int32_t* kind, int32_t* skip) {
  if (!spec || !kind || !skip) return DCG_ERR_ARG;
  const std::string sp(spec);
  const size_t colon = sp.find(':');
  const std::string name = sp.substr(0, colon);
  int32_t k = -1;
  if (name == "none" || name.empty()) k = DCG_FAULT_NONE;
  else if (name == "h2d_fail") k = DCG_FAULT_H2D_FAIL;
  else if (name == "short_copy") k = DCG_FAULT_SHORT_COPY;
  else if (name == "budget") k = DCG_FAULT_BUDGET;
  if (k < 0) return DCG_ERR_ARG;
  long n = 0;
  if (colon != std::string::npos) {
    const std::string rest = sp.substr(colon + 1);
    if (rest.empty() || rest.size() > 9 || rest.find_first_not_of("0123456789") != std::string::npos) return DCG_ERR_ARG;
    n = std::stol(rest);
  }
  *kind = k;
  *skip = (int32_t)n;
  return DCG_OK;
}

dcg_status dcg_inject_fault(dcg_ctx* ctx, int32_t kind, int32_t skip) {
  if (!ctx || kind < DCG_FAULT_NONE || kind > DCG_FAULT_BUDGET || skip < 0) return DCG_ERR_ARG;
  ctx->fault_kind = kind;
  ctx->fault_skip = skip;
  if (kind == DCG_FAULT_SHORT_COPY) ctx->verify_loads = true;  // the checksum is what detects it
  return DCG_OK;
}

dcg_status dcg_sync(dcg_ctx* ctx, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(ctx->h_errword, ctx->d_errword, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaStreamSynchronize(ctx->copy_stream));
  const unsigned w = *ctx->h_errword;
  if (w) {
    CK(cudaMemsetAsync(ctx->d_errword, 0, sizeof(unsigned), s));
    CK(cudaStreamSynchronize(s));
    if (w & ERRW_KEY_RANGE_BIT) return fail(ctx, DCG_ERR_KEY_RANGE, "chunk coordinate outside [-2^20, 2^20-1]");
    if (w & ERRW_CAPACITY_BIT) return fail(ctx, DCG_ERR_CAPACITY, "instance capacity exceeded");
    if (w & ERRW_TIMEOUT_BIT) return fail(ctx, DCG_ERR_TIMEOUT, "bounded device wait gave up");
    if (w & ERRW_BOUNDS_BIT) return fail(ctx, DCG_ERR_BOUNDS, "index outside its buffer (access skipped)");
  }
  return DCG_OK;
}

// ---------------------------------------------------------------- chunks
dcg_status dcg_chunk_keys(dcg_ctx* ctx, const float* means, int64_t n, uint64_t* keys_out, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!means || !keys_out))) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  launch_chunk_keys(means, 3, 1, n, ctx->cfg.chunk_size, (u64*)keys_out, ctx->d_errword, ctx->num_sms,
                    (cudaStream_t)stream);
  CK(cudaGetLastError());
  return DCG_OK;
}

dcg_status dcg_chunk_table_update(dcg_ctx* ctx, const float* params, int64_t stride, int64_t n, uint64_t* keys_out,
                                  void* stream) {
  if (!ctx || n < 0 || (n > 0 && !params) || stride < n) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if (n == 0) return DCG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int F = ctx->F;
  {
    dcg_status wb = writeback_active(ctx, s);
    if (wb != DCG_OK) return wb;
    ctx->active_fresh = false;  // chunks may grow: the next gather copies again
  }
  if (n > ctx->keys_cap) {
    cudaFree(ctx->d_keys);
    if (ctx->h_keys) cudaFreeHost(ctx->h_keys);
    ctx->d_keys = nullptr;
    ctx->h_keys = nullptr;
    ctx->keys_cap = 0;
    CK(dmalloc(&ctx->d_keys, (size_t)n));
    CK(cudaHostAlloc((void**)&ctx->h_keys, sizeof(uint64_t) * (size_t)n, 0));
    ctx->keys_cap = n;
  }
  if (n * F > ctx->stage_cap) {
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->stage_cap = 0;
    CK(cudaHostAlloc((void**)&ctx->h_stage, sizeof(float) * (size_t)(n * F), 0));
    ctx->stage_cap = n * F;
  }
  // Eq. 5 / 6 on the device (planar means: component stride `stride`)
  launch_chunk_keys(params, 1, stride, n, ctx->cfg.chunk_size, (u64*)ctx->d_keys, ctx->d_errword, ctx->num_sms, s);
  CK(cudaGetLastError());
  if (keys_out) CK(cudaMemcpyAsync(keys_out, ctx->d_keys, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(ctx->h_keys, ctx->d_keys, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpy2DAsync(ctx->h_stage, (size_t)n * 4, params, (size_t)stride * 4, (size_t)n * 4, (size_t)F,
                       cudaMemcpyDeviceToHost, s));
  dcg_status es = dcg_sync(ctx, stream);
  if (es != DCG_OK) return es;
  // group by chunk, stable in input order
  std::unordered_map<uint64_t, std::vector<int64_t>> groups;
  for (int64_t i = 0; i < n; ++i) groups[ctx->h_keys[i]].push_back(i);
  std::vector<uint64_t> new_keys;
  for (auto& kv : groups)
    if (!ctx->index.count(kv.first)) new_keys.push_back(kv.first);
  if ((int64_t)(ctx->chunks.size() + new_keys.size()) > ctx->cfg.max_chunks)
    return fail(ctx, DCG_ERR_CAPACITY, "chunk table full");
  int64_t need_pages = 0;
  for (auto& kv : groups) {
    int64_t have = 0, cnt0 = 0;
    auto it = ctx->index.find(kv.first);
    if (it != ctx->index.end()) {
      have = (int64_t)ctx->chunks[it->second].host_pages.size();
      cnt0 = ctx->chunks[it->second].count;
    }
    need_pages += pages_for(ctx, cnt0 + (int64_t)kv.second.size()) - have;
  }
  if (need_pages > (int64_t)ctx->host_free.size()) return fail(ctx, DCG_ERR_CAPACITY, "host tier full");
  // new chunks, table kept in ascending key order
  for (uint64_t k : new_keys) {
    Chunk ch;
    ch.key = k;
    const int64_t m = (1 << 21) - 1;
    ch.c[0] = (int32_t)((int64_t)((k >> 42) & m) - (1 << 20));
    ch.c[1] = (int32_t)((int64_t)((k >> 21) & m) - (1 << 20));
    ch.c[2] = (int32_t)((int64_t)(k & m) - (1 << 20));
    ctx->chunks.push_back(ch);
  }
  if (!new_keys.empty()) {
    std::sort(ctx->chunks.begin(), ctx->chunks.end(), [](const Chunk& a, const Chunk& b) { return a.key < b.key; });
    ctx->index.clear();
    for (size_t k = 0; k < ctx->chunks.size(); ++k) ctx->index[ctx->chunks[k].key] = (int32_t)k;
    dcg_status us = upload_coords(ctx);
    if (us != DCG_OK) return us;
  }
  CK(cudaStreamSynchronize(ctx->copy_stream));
  for (auto& kv : groups) {
    Chunk& ch = ctx->chunks[ctx->index[kv.first]];
    if (ch.resident) {  // write back and drop: the next gather reloads the whole chunk
      dcg_status e = evict_chunk(ctx, ch);
      if (e != DCG_OK) return e;
      ctx->evictions--;
      CK(cudaStreamSynchronize(ctx->copy_stream));
    }
    for (int64_t i : kv.second) {
      const int64_t slot = ch.count;
      const int64_t p = slot / ctx->page_g, j = slot - p * ctx->page_g;
      if (p >= (int64_t)ch.host_pages.size()) {
        ch.host_pages.push_back(ctx->host_free.back());
        ctx->host_free.pop_back();
      }
      float* page = host_page(ctx, ch.host_pages[(size_t)p]);
      for (int f = 0; f < F; ++f) page[(int64_t)f * ctx->page_g + j] = ctx->h_stage[(int64_t)f * n + i];
      for (int f = F; f < ctx->Fs; ++f) page[(int64_t)f * ctx->page_g + j] = 0.f;  // fresh Adam moments
      ch.count++;
    }
  }
  return DCG_OK;
}

int32_t dcg_chunk_count(const dcg_ctx* ctx) { return ctx ? (int32_t)ctx->chunks.size() : 0; }

dcg_status dcg_chunk_info(const dcg_ctx* ctx, int32_t* coords, uint64_t* keys, int64_t* counts, uint8_t* resident,
                          int64_t* last_access) {
  if (!ctx) return DCG_ERR_ARG;
  for (size_t k = 0; k < ctx->chunks.size(); ++k) {
    const Chunk& ch = ctx->chunks[k];
    if (coords)
      for (int a = 0; a < 3; ++a) coords[3 * k + a] = ch.c[a];
    if (keys) keys[k] = ch.key;
    if (counts) counts[k] = ch.count;
    if (resident) resident[k] = ch.resident ? 1 : 0;
    if (last_access) last_access[k] = ch.last_access;
  }
  return DCG_OK;
}

dcg_status dcg_cull_chunks(dcg_ctx* ctx, const dcg_camera* cams, int32_t n_views, uint8_t* mask_out, int32_t* list_out,
                           int32_t* n_out, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  dcg_status cs = check_cams(ctx, cams, n_views);
  if (cs != DCG_OK) return cs;
  // The cull reads only the chunk table (uploaded synchronously), so without a
  // mask to order against the caller's stream it runs on the context's own
  // stream and the host waits for that alone, not for the caller's queued work.
  // With the phase timers on it stays on the caller's stream, so that its
  // interval times the cull and not its wait for SMs busy with queued work.
  cudaStream_t s = (mask_out || ctx->prof_on) ? (cudaStream_t)stream : ctx->cull_stream;
  const int C = (int)ctx->chunks.size();
  std::memcpy(ctx->h_cullcams, cams, sizeof(dcg_camera) * n_views);
  CK(cudaMemcpyAsync(ctx->d_cullcams, ctx->h_cullcams, sizeof(dcg_camera) * n_views, cudaMemcpyHostToDevice, s));
  hook(ctx)(PH_CULL, true, s);
  CK(launch_cull(ctx->d_coords, C, ctx->d_cullcams, nullptr, n_views, ctx->cfg.chunk_size, ctx->cfg.dfar, mask_out,
                 ctx->d_vis, ctx->d_list, ctx->d_nlist, s));
  hook(ctx)(PH_CULL, false, s);
  CK(cudaMemcpyAsync(ctx->h_nlist, ctx->d_nlist, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (C > 0) CK(cudaMemcpyAsync(ctx->h_list, ctx->d_list, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (n_out) *n_out = *ctx->h_nlist;
  if (list_out) std::memcpy(list_out, ctx->h_list, sizeof(int32_t) * (size_t)*ctx->h_nlist);
  return DCG_OK;
}

// Compares every pending load check (verification mode) with the checksum of
// the pages that arrived.  A chunk that fails is dropped from the device (its
// pages freed, not written back), so the next gather loads it again.
dcg_status check_loads(dcg_ctx* ctx) {
  if (ctx->load_checks.empty()) return DCG_OK;
  const size_t n = ctx->load_checks.size();
  CK(cudaMemcpyAsync(ctx->h_loadsum, ctx->d_loadsum, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost,
                     ctx->copy_stream));
  CK(cudaStreamSynchronize(ctx->copy_stream));
  int bad = 0;
  for (size_t k = 0; k < n; ++k) {
    if (ctx->h_loadsum[k] == ctx->load_checks[k].second) continue;
    auto it = ctx->index.find(ctx->load_checks[k].first);
    if (it == ctx->index.end()) continue;
    Chunk& ch = ctx->chunks[(size_t)it->second];
    if (!ch.resident) continue;
    for (int32_t p : ch.dev_pages) ctx->dev_free.push_back(p);
    ch.dev_pages.clear();
    ch.resident = false;
    ch.dirty = false;
    ctx->resident_g -= ch.count;
    ++bad;
  }
  ctx->load_checks.clear();
  if (bad) return fail(ctx, DCG_ERR_FAULT, std::to_string(bad) + " chunk load(s) failed verification (dropped)");
  return DCG_OK;
}

dcg_status dcg_cull_chunks_async(dcg_ctx* ctx, const dcg_camera* cams, int32_t n_views, uint8_t* mask_out,
                                 int32_t* list_out, int32_t* n_out, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  // up to 16 views, whatever the render capacity (max_views) of the context
  if (!cams || n_views <= 0 || n_views > kMaxViewsApi) return fail(ctx, DCG_ERR_ARG, "bad views");
  for (int v = 0; v < n_views; ++v) {
    const dcg_camera& c = cams[v];
    if (c.W <= 0 || c.H <= 0 || !(c.fx > 0) || !(c.fy > 0) || !(c.znear > 0) || !(c.zfar > c.znear))
      return fail(ctx, DCG_ERR_ARG, "bad camera");
  }
  if (!list_out || !n_out) return fail(ctx, DCG_ERR_ARG, "list_out and n_out are required");
  CullCams tab;
  std::memset(&tab, 0, sizeof(tab));
  std::memcpy(tab.c, cams, sizeof(dcg_camera) * n_views);
  cudaStream_t s = (cudaStream_t)stream;
  hook(ctx)(PH_CULL, true, s);
  CK(launch_cull(ctx->d_coords, (int)ctx->chunks.size(), nullptr, &tab, n_views, ctx->cfg.chunk_size, ctx->cfg.dfar,
                 mask_out, ctx->d_vis_async, list_out, n_out, s));
  hook(ctx)(PH_CULL, false, s);
  return DCG_OK;
}

dcg_status dcg_gather_active(dcg_ctx* ctx, const int32_t* list, int32_t n_list, dcg_gaussians* active_out,
                             int64_t* n_active_out, void* stream) {
  if (!ctx || n_list < 0 || (n_list > 0 && !list) || !active_out || !n_active_out)
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int C = (int)ctx->chunks.size();
  std::vector<uint8_t> need((size_t)C, 0);
  int64_t total = 0, incoming = 0, need_pages = 0;
  for (int k = 0; k < n_list; ++k) {
    const int32_t c = list[k];
    if (c < 0 || c >= C || (k > 0 && list[k - 1] >= c)) return fail(ctx, DCG_ERR_ARG, "chunk list must be ascending indices");
    need[(size_t)c] = 1;
    total += ctx->chunks[c].count;
    if (!ctx->chunks[c].resident) {
      incoming += ctx->chunks[c].count;
      need_pages += pages_for(ctx, ctx->chunks[c].count);
    }
  }
  if (total > ctx->cfg.device_budget || total > ctx->cfg.max_active)
    return fail(ctx, DCG_ERR_BUDGET, "visible chunks exceed the device budget");
  if (fault_fires(ctx, DCG_FAULT_BUDGET)) return fail(ctx, DCG_ERR_BUDGET, "injected budget failure");
  // the active buffer already holds exactly these chunks: hand it out again
  bool reuse = ctx->active_valid && ctx->active_fresh && (size_t)n_list == ctx->active_keys.size();
  for (int k = 0; reuse && k < n_list; ++k)
    reuse = ctx->chunks[list[k]].key == ctx->active_keys[(size_t)k] && ctx->chunks[list[k]].resident;
  if (reuse) {
    ctx->step++;
    for (int k = 0; k < n_list; ++k) ctx->chunks[list[k]].last_access = ctx->step;
    active_out->data = ctx->d_active;
    active_out->stride = ctx->cfg.max_active;
    active_out->sh_degree = ctx->cfg.sh_degree;
    active_out->pad = 0;
    *n_active_out = ctx->n_active;
    return DCG_OK;
  }
  {
    dcg_status wb = writeback_active(ctx, s);
    if (wb != DCG_OK) return wb;
  }
  ctx->step++;
  // LRU eviction (Sec. III-E): oldest first, ties by id, the fewest chunks that make room
  int64_t deficit_g = ctx->resident_g + incoming - ctx->cfg.device_budget;
  int64_t deficit_p = need_pages - (int64_t)ctx->dev_free.size();
  if (deficit_g > 0 || deficit_p > 0) {
    std::vector<int32_t> cand;
    for (int c = 0; c < C; ++c)
      if (ctx->chunks[c].resident && !need[(size_t)c]) cand.push_back(c);
    std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) {
      const Chunk &x = ctx->chunks[a], &y = ctx->chunks[b];
      return x.last_access < y.last_access || (x.last_access == y.last_access && x.key < y.key);
    });
    CK(cudaEventRecord(ctx->ev_compute, s));
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_compute, 0));
    for (int32_t c : cand) {
      if (deficit_g <= 0 && deficit_p <= 0) break;
      const int64_t cnt = ctx->chunks[c].count;
      const int64_t np = (int64_t)ctx->chunks[c].dev_pages.size();
      dcg_status e = evict_chunk(ctx, ctx->chunks[c]);
      if (e != DCG_OK) return e;
      deficit_g -= cnt;
      deficit_p -= np;
    }
    if (deficit_g > 0 || deficit_p > 0) return fail(ctx, DCG_ERR_BUDGET, "cannot make room within the budget");
  }
  // loads on the copy stream
  bool any_load = false;
  for (int k = 0; k < n_list; ++k) {
    Chunk& ch = ctx->chunks[list[k]];
    if (!ch.resident) {
      if (!any_load) {
        CK(cudaEventRecord(ctx->ev_compute, s));
        CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_compute, 0));
        any_load = true;
      }
      dcg_status e = load_chunk(ctx, ch);
      if (e != DCG_OK) return e;
    }
    ch.last_access = ctx->step;
  }
  {
    dcg_status vs = check_loads(ctx);
    if (vs != DCG_OK) return vs;
  }
  // wait only for the copies the listed chunks need: the copy stream is in
  // order, so the listed chunk loaded last stands for all of them (prefetches
  // of chunks not needed yet keep running)
  const Chunk* newest = nullptr;
  for (int k = 0; k < n_list; ++k) {
    const Chunk& ch = ctx->chunks[list[k]];
    if (ch.ev_load && (!newest || ch.load_seq > newest->load_seq)) newest = &ch;
  }
  hook(ctx)(PH_STALL, true, s);
  if (newest) CK(cudaStreamWaitEvent(s, newest->ev_load, 0));
  hook(ctx)(PH_STALL, false, s);
  // page descriptors: (page, count, offset in the active buffer)
  long long* hd = nullptr;
  {
    dcg_status ds = desc_stage(ctx, &hd);
    if (ds != DCG_OK) return ds;
  }
  int nd = 0;
  int64_t off = 0;
  ctx->active_keys.clear();
  ctx->active_counts.clear();
  for (int k = 0; k < n_list; ++k) {
    const Chunk& ch = ctx->chunks[list[k]];
    ctx->active_keys.push_back(ch.key);
    ctx->active_counts.push_back(ch.count);
    for (size_t p = 0; p < ch.dev_pages.size(); ++p) {
      const int64_t cnt = std::min<int64_t>(ctx->page_g, ch.count - (int64_t)p * ctx->page_g);
      hd[3 * nd + 0] = ch.dev_pages[p];
      hd[3 * nd + 1] = cnt;
      hd[3 * nd + 2] = off;
      off += cnt;
      ++nd;
    }
  }
  {
    dcg_status us = desc_upload(ctx, nd, s);
    if (us != DCG_OK) return us;
  }
  hook(ctx)(PH_GATHER, true, s);
  launch_page_copy(true, ctx->d_pool, ctx->page_g, ctx->Fs, 0, ctx->Fs, active_desc(ctx), nd, ctx->d_active,
                   ctx->cfg.max_active, s);
  hook(ctx)(PH_GATHER, false, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->ev_compute, s));
  ctx->n_active = total;
  ctx->active_valid = true;
  ctx->active_fresh = false;  // only a scatter_back of this buffer makes it reusable
  active_out->data = ctx->d_active;
  active_out->stride = ctx->cfg.max_active;
  active_out->sh_degree = ctx->cfg.sh_degree;
  active_out->pad = 0;
  *n_active_out = total;
  return DCG_OK;
}

dcg_status dcg_prefetch(dcg_ctx* ctx, const int32_t* list, int32_t n_list, int32_t* n_loaded, void* stream) {
  if (!ctx || n_list < 0 || (n_list > 0 && !list)) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if (n_loaded) *n_loaded = 0;
  const int C = (int)ctx->chunks.size();
  std::vector<uint8_t> keep((size_t)C, 0);
  for (int k = 0; k < n_list; ++k) {
    if (list[k] < 0 || list[k] >= C) return fail(ctx, DCG_ERR_ARG, "chunk index out of range");
    keep[(size_t)list[k]] = 1;
  }
  for (uint64_t key : ctx->active_keys) {
    auto it = ctx->index.find(key);
    if (it != ctx->index.end()) keep[(size_t)it->second] = 1;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // evictions below must follow the compute stream's use of the pages
  CK(cudaEventRecord(ctx->ev_compute, s));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_compute, 0));
  std::vector<int32_t> cand;
  for (int c = 0; c < C; ++c)
    if (ctx->chunks[c].resident && !keep[(size_t)c]) cand.push_back(c);
  std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) {
    const Chunk &x = ctx->chunks[a], &y = ctx->chunks[b];
    return x.last_access < y.last_access || (x.last_access == y.last_access && x.key < y.key);
  });
  size_t next_victim = 0;
  int32_t loaded = 0;
  for (int k = 0; k < n_list; ++k) {
    Chunk& ch = ctx->chunks[list[k]];
    if (ch.resident) continue;
    const int64_t np = pages_for(ctx, ch.count);
    while ((ctx->resident_g + ch.count > ctx->cfg.device_budget || (int64_t)ctx->dev_free.size() < np) &&
           next_victim < cand.size()) {
      dcg_status e = evict_chunk(ctx, ctx->chunks[cand[next_victim++]]);
      if (e != DCG_OK) return e;
    }
    if (ctx->resident_g + ch.count > ctx->cfg.device_budget || (int64_t)ctx->dev_free.size() < np) break;
    dcg_status e = load_chunk(ctx, ch);
    if (e != DCG_OK) return e;
    ch.last_access = ctx->step;
    ++loaded;
  }
  if (n_loaded) *n_loaded = loaded;
  return DCG_OK;
}

dcg_status dcg_chunks_near(const dcg_ctx* ctx, const float* p, float radius, int32_t only_nonresident,
                           int32_t* list_out, int32_t* n_out) {
  if (!ctx || !p || !list_out || !n_out) return DCG_ERR_ARG;
  const double s = ctx->cfg.chunk_size, r2 = (double)radius * radius;
  int32_t k = 0;
  for (size_t c = 0; c < ctx->chunks.size(); ++c) {
    const Chunk& ch = ctx->chunks[c];
    if (only_nonresident && ch.resident) continue;
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double lo = ch.c[a] * s - 0.5 * s, hi = ch.c[a] * s + 0.5 * s;
      const double e = p[a] < lo ? lo - p[a] : (p[a] > hi ? p[a] - hi : 0.0);
      d2 += e * e;
    }
    if (d2 <= r2) list_out[k++] = (int32_t)c;
  }
  *n_out = k;
  return DCG_OK;
}

dcg_status dcg_tier_stats(const dcg_ctx* ctx, int64_t* loads, int64_t* evictions, int64_t* bytes_h2d,
                          int64_t* bytes_d2h, int64_t* resident) {
  if (!ctx) return DCG_ERR_ARG;
  if (loads) *loads = ctx->loads;
  if (evictions) *evictions = ctx->evictions;
  if (bytes_h2d) *bytes_h2d = ctx->bytes_h2d;
  if (bytes_d2h) *bytes_d2h = ctx->bytes_d2h;
  if (resident) *resident = ctx->resident_g;
  return DCG_OK;
}

dcg_status dcg_scatter_back(dcg_ctx* ctx, const dcg_gaussians* active, int64_t n, void* stream) {
  if (!ctx || !active || !active->data) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if (!ctx->active_valid) return fail(ctx, DCG_ERR_STATE, "scatter_back without a gather");
  if (n != ctx->n_active || active->sh_degree != ctx->cfg.sh_degree || active->stride < n)
    return fail(ctx, DCG_ERR_ARG, "scatter_back size or degree differs from the gather");
  cudaStream_t s = (cudaStream_t)stream;
  for (uint64_t k : ctx->active_keys) {
    auto it = ctx->index.find(k);
    if (it == ctx->index.end() || !ctx->chunks[it->second].resident)
      return fail(ctx, DCG_ERR_STATE, "a gathered chunk is no longer resident");
  }
  hook(ctx)(PH_SCATTER, true, s);
  if (active->data == ctx->d_active && active->stride == ctx->cfg.max_active) {
    // the active buffer itself: the copy to the pages is deferred (write-back)
    ctx->active_dirty = true;
    ctx->active_fresh = true;
  } else {  // parameters from the caller's buffer, moments from the active buffer
    ctx->active_dirty = false;
    ctx->active_fresh = false;
    launch_page_copy(false, ctx->d_pool, ctx->page_g, ctx->Fs, 0, ctx->F, active_desc(ctx), ctx->n_desc, active->data,
                     active->stride, s);
    if (ctx->Fs > ctx->F)
      launch_page_copy(false, ctx->d_pool, ctx->page_g, ctx->Fs, ctx->F, ctx->Fs - ctx->F, active_desc(ctx), ctx->n_desc,
                       ctx->d_active + (size_t)ctx->F * ctx->cfg.max_active, ctx->cfg.max_active, s);
  }
  hook(ctx)(PH_SCATTER, false, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->ev_compute, s));
  for (uint64_t k : ctx->active_keys) ctx->chunks[ctx->index[k]].dirty = true;
  return DCG_OK;
}

dcg_status dcg_active_map(dcg_ctx* ctx, int32_t* chunk_out, int32_t* row_out, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  if (!ctx->active_valid) return fail(ctx, DCG_ERR_STATE, "no gathered active set");
  const int nl = (int)ctx->active_keys.size();
  if (nl == 0 || ctx->n_active == 0 || (!chunk_out && !row_out)) return DCG_OK;
  // the staging buffers are free once the previous call's upload has run
  CK(cudaEventSynchronize(ctx->ev_am));
  long long o = 0;
  for (int k = 0; k < nl; ++k) {
    auto it = ctx->index.find(ctx->active_keys[(size_t)k]);
    if (it == ctx->index.end()) return fail(ctx, DCG_ERR_STATE, "a gathered chunk left the table");
    ctx->h_amchunk[k] = it->second;
    ctx->h_amoff[k] = o;
    o += ctx->active_counts[(size_t)k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(ctx->d_amoff, ctx->h_amoff, sizeof(long long) * (size_t)nl, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->d_amchunk, ctx->h_amchunk, sizeof(int32_t) * (size_t)nl, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(ctx->ev_am, s));
  launch_active_map(ctx->d_amoff, ctx->d_amchunk, nl, ctx->n_active, chunk_out, row_out, ctx->num_sms, s);
  CK(cudaGetLastError());
  return DCG_OK;
}

dcg_status dcg_flush(dcg_ctx* ctx, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  {
    dcg_status wb = writeback_active(ctx, s);
    if (wb != DCG_OK) return wb;
  }
  CK(cudaEventRecord(ctx->ev_compute, s));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_compute, 0));
  for (Chunk& ch : ctx->chunks) {
    if (!ch.resident || !ch.dirty) continue;
    for (size_t p = 0; p < ch.dev_pages.size(); ++p) {
      const int64_t cnt = std::min<int64_t>(ctx->page_g, ch.count - (int64_t)p * ctx->page_g);
      CK(page_copy(ctx, host_page(ctx, ch.host_pages[p]), dev_page(ctx, ch.dev_pages[p]), cnt, cudaMemcpyDeviceToHost,
                   ctx->copy_stream));
      ctx->bytes_d2h += cnt * ctx->Fs * 4;
    }
    ch.dirty = false;
  }
  CK(cudaStreamSynchronize(ctx->copy_stream));
  return DCG_OK;
}

dcg_status dcg_chunk_read(dcg_ctx* ctx, int32_t chunk, float* out, int64_t n) {
  if (!ctx || chunk < 0 || chunk >= (int32_t)ctx->chunks.size() || !out) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  const Chunk& ch = ctx->chunks[chunk];
  if (n != ch.count) return fail(ctx, DCG_ERR_ARG, "n must equal the chunk's count");
  CK(cudaStreamSynchronize(ctx->copy_stream));
  for (int64_t i = 0; i < n; ++i) {
    const int64_t p = i / ctx->page_g, j = i - p * ctx->page_g;
    const float* page = host_page(ctx, ch.host_pages[(size_t)p]);
    for (int f = 0; f < ctx->F; ++f) out[(int64_t)f * n + i] = page[(int64_t)f * ctx->page_g + j];
  }
  return DCG_OK;
}

dcg_status dcg_chunk_read_moments(dcg_ctx* ctx, int32_t chunk, float* m_out, float* v_out, int64_t n) {
  if (!ctx || chunk < 0 || chunk >= (int32_t)ctx->chunks.size() || !m_out || !v_out)
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if (ctx->Fs == ctx->F) return fail(ctx, DCG_ERR_ARG, "the context stores no optimizer moments");
  const Chunk& ch = ctx->chunks[chunk];
  if (n != ch.count) return fail(ctx, DCG_ERR_ARG, "n must equal the chunk's count");
  CK(cudaStreamSynchronize(ctx->copy_stream));
  const int F = ctx->F;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t p = i / ctx->page_g, j = i - p * ctx->page_g;
    const float* page = host_page(ctx, ch.host_pages[(size_t)p]);
    for (int f = 0; f < F; ++f) {
      m_out[(int64_t)f * n + i] = page[(int64_t)(F + f) * ctx->page_g + j];
      v_out[(int64_t)f * n + i] = page[(int64_t)(2 * F + f) * ctx->page_g + j];
    }
  }
  return DCG_OK;
}

// ---------------------------------------------------------------- optimizer
dcg_status dcg_active_moments(dcg_ctx* ctx, dcg_gaussians* m, dcg_gaussians* v) {
  if (!ctx || !m || !v) return DCG_ERR_ARG;
  if (ctx->Fs == ctx->F) return fail(ctx, DCG_ERR_ARG, "the context stores no optimizer moments");
  const int64_t S = ctx->cfg.max_active;
  m->data = ctx->d_active + (size_t)ctx->F * S;
  v->data = ctx->d_active + (size_t)2 * ctx->F * S;
  m->stride = v->stride = S;
  m->sh_degree = v->sh_degree = ctx->cfg.sh_degree;
  m->pad = v->pad = 0;
  return DCG_OK;
}

dcg_status dcg_adam_step(dcg_ctx* ctx, const dcg_gaussians* params, const dcg_gaussians* grads, int64_t n,
                         const float* lr, float beta1, float beta2, float eps, int64_t step, void* stream) {
  if (!ctx || !params || !grads || !lr || !params->data || !grads->data) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if (ctx->Fs == ctx->F) return fail(ctx, DCG_ERR_ARG, "the context stores no optimizer moments");
  if (!ctx->active_valid || n != ctx->n_active) return fail(ctx, DCG_ERR_STATE, "n must equal the gathered active set");
  if (params->sh_degree != ctx->cfg.sh_degree || grads->sh_degree != ctx->cfg.sh_degree || params->stride < n ||
      grads->stride < n)
    return fail(ctx, DCG_ERR_ARG, "degree or stride does not match the active set");
  if (step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return fail(ctx, DCG_ERR_ARG, "bad Adam hyper-parameters");
  const int F = ctx->F;
  if (F > kAdamMaxF) return fail(ctx, DCG_ERR_ARG, "too many components");
  AdamArgs aa{};
  const double bc1 = 1.0 - std::pow((double)beta1, (double)step), bc2 = 1.0 - std::pow((double)beta2, (double)step);
  for (int c = 0; c < F; ++c) {
    if (!std::isfinite(lr[c])) return fail(ctx, DCG_ERR_ARG, "learning rate not finite");
    aa.step[c] = (float)(lr[c] / bc1);
  }
  aa.beta1 = beta1;
  aa.beta2 = beta2;
  aa.isb2 = (float)(1.0 / std::sqrt(bc2));
  aa.eps = eps;
  const int64_t S = ctx->cfg.max_active;
  launch_adam(params->data, params->stride, grads->data, grads->stride, ctx->d_active + (size_t)F * S,
              ctx->d_active + (size_t)2 * F * S, S, n, F, aa, ctx->num_sms, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return DCG_OK;
}

// ---------------------------------------------------------------- loop closure
// Unit quaternion (w, x, y, z) of a rotation matrix (row-major), Shepperd's method.
static void rot_to_quat(const double R[9], double q[4]) {
  const double tr = R[0] + R[4] + R[8];
  if (tr > 0.0) {
    const double s = 2.0 * std::sqrt(1.0 + tr);
    q[0] = 0.25 * s;
    q[1] = (R[7] - R[5]) / s;
    q[2] = (R[2] - R[6]) / s;
    q[3] = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const double s = 2.0 * std::sqrt(1.0 + R[0] - R[4] - R[8]);
    q[0] = (R[7] - R[5]) / s;
    q[1] = 0.25 * s;
    q[2] = (R[1] + R[3]) / s;
    q[3] = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const double s = 2.0 * std::sqrt(1.0 + R[4] - R[0] - R[8]);
    q[0] = (R[2] - R[6]) / s;
    q[1] = (R[1] + R[3]) / s;
    q[2] = 0.25 * s;
    q[3] = (R[5] + R[7]) / s;
  } else {
    const double s = 2.0 * std::sqrt(1.0 + R[8] - R[0] - R[4]);
    q[0] = (R[3] - R[1]) / s;
    q[1] = (R[2] + R[6]) / s;
    q[2] = (R[5] + R[7]) / s;
    q[3] = 0.25 * s;
  }
  const double l = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] /= l;
}

// Appends Gaussian j of the planar host rows (`rows` components, stride
// `stride`) to chunk ch in the host tier; components >= rows are zeroed.
static void append_host_row(dcg_ctx* ctx, Chunk& ch, const float* src, int64_t stride, int64_t j, int rows) {
  const int64_t slot = ch.count;
  const int64_t p = slot / ctx->page_g, o = slot - p * ctx->page_g;
  if (p >= (int64_t)ch.host_pages.size()) {
    ch.host_pages.push_back(ctx->host_free.back());
    ctx->host_free.pop_back();
  }
  float* page = host_page(ctx, ch.host_pages[(size_t)p]);
  for (int f = 0; f < rows; ++f) page[(int64_t)f * ctx->page_g + o] = src[(int64_t)f * stride + j];
  for (int f = rows; f < ctx->Fs; ++f) page[(int64_t)f * ctx->page_g + o] = 0.f;
  ch.count++;
}

static Chunk make_chunk(uint64_t k) {
  Chunk ch;
  ch.key = k;
  const int64_t m = (1 << 21) - 1;
  ch.c[0] = (int32_t)((int64_t)((k >> 42) & m) - (1 << 20));
  ch.c[1] = (int32_t)((int64_t)((k >> 21) & m) - (1 << 20));
  ch.c[2] = (int32_t)((int64_t)(k & m) - (1 << 20));
  return ch;
}

// Device scratch of a loop closure over n gathered Gaussians, kept between
// calls and grown on demand (a loop closure is a rare event, not a render step).
static dcg_status lc_reserve(dcg_ctx* ctx, int64_t n, cudaStream_t s) {
  if (n <= ctx->lc_dev_cap) return DCG_OK;
  const int Fs = ctx->Fs;
  CK(cudaStreamSynchronize(s));
  cudaFree(ctx->d_lctmp);
  cudaFree(ctx->d_lcperm);
  cudaFree(ctx->d_lcmidx);
  cudaFree(ctx->d_lcmkey);
  ctx->d_lctmp = nullptr;
  ctx->d_lcperm = ctx->d_lcmidx = nullptr;
  ctx->d_lcmkey = nullptr;
  ctx->lc_dev_cap = 0;
  CK(cudaMalloc((void**)&ctx->d_lctmp, sizeof(float) * (size_t)Fs * (size_t)n));
  CK(cudaMalloc((void**)&ctx->d_lcperm, sizeof(long long) * (size_t)n));
  CK(cudaMalloc((void**)&ctx->d_lcmidx, sizeof(long long) * (size_t)n));
  CK(cudaMalloc((void**)&ctx->d_lcmkey, sizeof(u64) * (size_t)n));
  ctx->lc_dev_cap = n;
  return DCG_OK;
}

// Drops the device copy of a chunk that is not dirty (its pages are freed).
static void drop_resident(dcg_ctx* ctx, Chunk& ch) {
  if (!ch.resident) return;
  for (int32_t p : ch.dev_pages) ctx->dev_free.push_back(p);
  ch.dev_pages.clear();
  ch.resident = false;
  ch.dirty = false;
  ctx->resident_g -= ch.count;
}

// The keyframe-by-keyframe order of Sec. III-F, for when the union of the
// affected keyframes' chunks does not fit the device budget: the keyframes
// are taken one at a time in the given order, each loading only the chunks
// its own cull keeps.  A Gaussian is tested against keyframe k at its
// uncorrected position unless an earlier keyframe has moved it: that global
// transformation mask persists across the loads as one flag per (chunk, row)
// on the host (rows keep their places until the end).  Every keyframe's
// corrections and moved rows are recorded on the host and applied to the
// host tier at the end, in the order the batch load produces (remaining
// rows in stored order, then the incoming ones by source chunk id and row),
// so the result equals the batch result; nothing changes before the last
// keyframe has been processed (a position outside the key range leaves the
// table as it was).  hmask: [K][C] cull of each keyframe.
static dcg_status loop_closure_by_keyframe(dcg_ctx* ctx, const uint8_t* hmask, int K, int C, int64_t* n_transformed,
                                           int64_t* n_moved, cudaStream_t s) {
  const int64_t cap = std::min<int64_t>(ctx->cfg.device_budget, ctx->cfg.max_active);
  std::vector<std::vector<int32_t>> lists((size_t)K);
  for (int k = 0; k < K; ++k) {
    int64_t total = 0;
    for (int c = 0; c < C; ++c)
      if (hmask[(size_t)k * C + c]) {
        lists[(size_t)k].push_back(c);
        total += ctx->chunks[(size_t)c].count;
      }
    if (total > cap) return fail(ctx, DCG_ERR_BUDGET, "the chunks of one keyframe exceed the device budget");
  }
  const int Fs = ctx->Fs;
  const int64_t S = ctx->cfg.max_active;
  dcg_render_state* st = ctx->st0;
  uint32_t* d_flags = st->touched;  // render scratch, at least max_active entries
  u64* d_keys = st->list_a;
  std::vector<std::vector<uint8_t>> done((size_t)C);  // the global transformation mask
  struct TRow {
    int32_t c;
    int64_t r;
    float v[7];  // corrected mean and quaternion
  };
  struct MRow {
    int32_t c;
    int64_t r;
    uint64_t key;  // chunk id of the corrected position
  };
  std::vector<TRow> trows;
  std::vector<MRow> mrows;
  int64_t nt = 0;
  std::vector<uint32_t> hflags;
  std::vector<float> hval;
  std::vector<long long> midx;
  std::vector<uint64_t> mkey;
  for (int k = 0; k < K; ++k) {
    const std::vector<int32_t>& lk = lists[(size_t)k];
    if (lk.empty()) continue;
    const int nl = (int)lk.size();
    dcg_gaussians g{};
    int64_t n = 0;
    dcg_status gs = dcg_gather_active(ctx, lk.data(), nl, &g, &n, s);
    if (gs != DCG_OK) return gs;
    ctx->active_valid = false;  // worked on in place below and never written back
    if (n == 0) continue;
    dcg_status rs = lc_reserve(ctx, n, s);
    if (rs != DCG_OK) return rs;
    std::vector<long long> seg((size_t)nl);
    std::vector<int> segc((size_t)nl);
    std::vector<uint64_t> segkey((size_t)nl);
    hflags.assign((size_t)n, 0u);
    long long off = 0;
    for (int j = 0; j < nl; ++j) {
      const Chunk& ch = ctx->chunks[(size_t)lk[(size_t)j]];
      seg[(size_t)j] = off;
      segc[(size_t)j] = lk[(size_t)j];
      segkey[(size_t)j] = ch.key;
      const std::vector<uint8_t>& dn = done[(size_t)lk[(size_t)j]];
      for (size_t r = 0; r < dn.size(); ++r) hflags[(size_t)off + r] = dn[r];
      off += ch.count;
    }
    CK(cudaMemcpyAsync(ctx->d_lcseg, seg.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_lcsegc, segc.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_lcsegkey, segkey.data(), sizeof(u64) * nl, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_flags, hflags.data(), sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    hook(ctx)(PH_LOOP, true, s);
    launch_loop_transform(ctx->d_active, S, n, ctx->d_lcseg, ctx->d_lcsegc, nl, ctx->d_lcmask + (size_t)k * C, C,
                          ctx->d_lcview + k, 1, d_flags, 1, ctx->num_sms, s);
    launch_chunk_keys(ctx->d_active, 1, S, n, ctx->cfg.chunk_size, d_keys, ctx->d_errword, ctx->num_sms, s);
    hook(ctx)(PH_LOOP, false, s);
    CK(cudaGetLastError());
    // the rows this keyframe moved, and the corrected mean and rotation of every row
    CK(cudaMemcpyAsync(hflags.data(), d_flags, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    hval.resize((size_t)7 * n);
    CK(cudaMemcpy2DAsync(hval.data(), (size_t)n * 4, ctx->d_active, (size_t)S * 4, (size_t)n * 4, 3,
                         cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpy2DAsync(hval.data() + 3 * n, (size_t)n * 4, ctx->d_active + 6 * S, (size_t)S * 4, (size_t)n * 4, 4,
                         cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(ctx->d_lccnt, 0, 2 * sizeof(u64), s));
    hook(ctx)(PH_LOOP, true, s);
    launch_lc_moved(d_flags, d_keys, n, ctx->d_lcseg, ctx->d_lcsegkey, nl, (unsigned long long*)ctx->d_lccnt,
                    ctx->d_lcmidx, ctx->d_lcmkey, st->part, st->P, ctx->d_lccnt + 1, ctx->num_sms, s);
    hook(ctx)(PH_LOOP, false, s);
    CK(cudaGetLastError());
    u64 cnt[2] = {0, 0};
    CK(cudaMemcpyAsync(cnt, ctx->d_lccnt, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    dcg_status es = dcg_sync(ctx, s);  // a position outside the key range stops here; nothing has changed yet
    if (es != DCG_OK) return es;
    const int64_t nm = (int64_t)cnt[1];
    midx.resize((size_t)nm);
    mkey.resize((size_t)nm);
    if (nm > 0) {
      CK(cudaMemcpyAsync(midx.data(), ctx->d_lcmidx, sizeof(long long) * (size_t)nm, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(mkey.data(), ctx->d_lcmkey, sizeof(u64) * (size_t)nm, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    for (int j = 0; j < nl; ++j) {
      const int32_t c = lk[(size_t)j];
      const int64_t cntc = ctx->chunks[(size_t)c].count;
      std::vector<uint8_t>& dn = done[(size_t)c];
      for (int64_t r = 0; r < cntc; ++r) {
        const int64_t i = seg[(size_t)j] + r;
        if (!hflags[(size_t)i]) continue;
        if (dn.empty()) dn.assign((size_t)cntc, 0);
        dn[(size_t)r] = 1;
        TRow t;
        t.c = c;
        t.r = r;
        for (int q = 0; q < 7; ++q) t.v[q] = hval[(size_t)q * n + i];
        trows.push_back(t);
      }
    }
    for (int64_t m = 0; m < nm; ++m) {
      const long long i = midx[(size_t)m];
      const int j = (int)(std::upper_bound(seg.begin(), seg.end(), i) - seg.begin()) - 1;
      mrows.push_back({lk[(size_t)j], (int64_t)(i - seg[(size_t)j]), mkey[(size_t)m]});
    }
    nt += (int64_t)cnt[0];
  }
  // apply, with the host tier as the stored value of every chunk
  {
    dcg_status fs = dcg_flush(ctx, s);
    if (fs != DCG_OK) return fs;
  }
  std::sort(mrows.begin(), mrows.end(), [](const MRow& a, const MRow& b) { return a.c < b.c || (a.c == b.c && a.r < b.r); });
  const int64_t nm = (int64_t)mrows.size();
  std::vector<int64_t> out_c((size_t)C, 0);
  std::map<uint64_t, int64_t> in_key;
  for (const MRow& m : mrows) {
    ++out_c[(size_t)m.c];
    ++in_key[m.key];
  }
  int64_t host_need = 0, new_chunks = 0;
  for (int c = 0; c < C; ++c) {
    const Chunk& ch = ctx->chunks[(size_t)c];
    auto it = in_key.find(ch.key);
    const int64_t in = it == in_key.end() ? 0 : it->second;
    if (out_c[(size_t)c] || in) host_need += pages_for(ctx, ch.count - out_c[(size_t)c] + in) - (int64_t)ch.host_pages.size();
  }
  for (auto& kv : in_key)
    if (!ctx->index.count(kv.first)) {
      ++new_chunks;
      host_need += pages_for(ctx, kv.second);
    }
  if (host_need > (int64_t)ctx->host_free.size()) return fail(ctx, DCG_ERR_CAPACITY, "host tier full");
  if ((int64_t)ctx->chunks.size() + new_chunks > ctx->cfg.max_chunks)
    return fail(ctx, DCG_ERR_CAPACITY, "chunk table full");
  // device copies of every chunk that changes are dropped (clean after the flush)
  for (const TRow& t : trows) drop_resident(ctx, ctx->chunks[(size_t)t.c]);
  for (auto& kv : in_key) {
    auto it = ctx->index.find(kv.first);
    if (it != ctx->index.end()) drop_resident(ctx, ctx->chunks[(size_t)it->second]);
  }
  // 1. the rigid corrections, in place
  static const int kComp[7] = {0, 1, 2, 6, 7, 8, 9};
  for (const TRow& t : trows) {
    const Chunk& ch = ctx->chunks[(size_t)t.c];
    const int64_t p = t.r / ctx->page_g, o = t.r - p * ctx->page_g;
    float* page = host_page(ctx, ch.host_pages[(size_t)p]);
    for (int q = 0; q < 7; ++q) page[(int64_t)kComp[q] * ctx->page_g + o] = t.v[q];
  }
  // 2. the moved rows' contents (planar [Fs][nm], gather order), then the
  // sources keep their remaining rows in stored order
  std::vector<float> mdata((size_t)Fs * (size_t)std::max<int64_t>(nm, 1));
  for (int64_t m = 0; m < nm; ++m) {
    const Chunk& ch = ctx->chunks[(size_t)mrows[(size_t)m].c];
    const int64_t r = mrows[(size_t)m].r, p = r / ctx->page_g, o = r - p * ctx->page_g;
    const float* page = host_page(ctx, ch.host_pages[(size_t)p]);
    for (int f = 0; f < Fs; ++f) mdata[(size_t)f * nm + m] = page[(int64_t)f * ctx->page_g + o];
  }
  {
    int64_t m = 0;
    std::vector<float> tmp;
    while (m < nm) {
      const int32_t c = mrows[(size_t)m].c;
      Chunk& ch = ctx->chunks[(size_t)c];
      tmp.assign((size_t)Fs * ch.count, 0.f);
      for (int64_t r = 0; r < ch.count; ++r) {
        const int64_t p = r / ctx->page_g, o = r - p * ctx->page_g;
        const float* page = host_page(ctx, ch.host_pages[(size_t)p]);
        for (int f = 0; f < Fs; ++f) tmp[(size_t)f * ch.count + r] = page[(int64_t)f * ctx->page_g + o];
      }
      const int64_t old = ch.count;
      int64_t w = 0;
      for (int64_t r = 0; r < old; ++r) {
        if (m < nm && mrows[(size_t)m].c == c && mrows[(size_t)m].r == r) {
          ++m;
          continue;
        }
        const int64_t p = w / ctx->page_g, o = w - p * ctx->page_g;
        float* page = host_page(ctx, ch.host_pages[(size_t)p]);
        for (int f = 0; f < Fs; ++f) page[(int64_t)f * ctx->page_g + o] = tmp[(size_t)f * old + r];
        ++w;
      }
      ch.count = w;
      ch.dirty = false;
      while ((int64_t)ch.host_pages.size() > pages_for(ctx, ch.count)) {
        ctx->host_free.push_back(ch.host_pages.back());
        ch.host_pages.pop_back();
      }
    }
  }
  // 3. the destinations receive the incoming rows after their own, in gather order
  bool added = false;
  for (int64_t m = 0; m < nm; ++m) {
    const uint64_t key = mrows[(size_t)m].key;
    auto it = ctx->index.find(key);
    if (it == ctx->index.end()) {
      ctx->chunks.push_back(make_chunk(key));
      ctx->index[key] = (int32_t)ctx->chunks.size() - 1;
      it = ctx->index.find(key);
      added = true;
    }
    append_host_row(ctx, ctx->chunks[(size_t)it->second], mdata.data(), nm, m, Fs);
  }
  if (added) {
    std::sort(ctx->chunks.begin(), ctx->chunks.end(), [](const Chunk& a, const Chunk& b) { return a.key < b.key; });
    ctx->index.clear();
    for (size_t k = 0; k < ctx->chunks.size(); ++k) ctx->index[ctx->chunks[k].key] = (int32_t)k;
    dcg_status us = upload_coords(ctx);
    if (us != DCG_OK) return us;
  }
  ctx->active_valid = false;
  ctx->active_fresh = false;
  ctx->active_dirty = false;
  if (n_transformed) *n_transformed = nt;
  if (n_moved) *n_moved = nm;
  return DCG_OK;
}

dcg_status dcg_loop_closure(dcg_ctx* ctx, const dcg_camera* kf, const float* corr, int32_t K, int64_t* n_transformed,
                            int64_t* n_moved, void* stream) {
  if (!ctx || !kf || !corr || K <= 0 || K > kMaxViewsApi) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  for (int k = 0; k < K; ++k) {
    const dcg_camera& c = kf[k];
    if (c.W <= 0 || c.H <= 0 || !(c.fx > 0.f) || !(c.fy > 0.f) || !(c.znear > 0.f) || !(c.zfar > c.znear))
      return fail(ctx, DCG_ERR_ARG, "bad keyframe camera");
    for (int e = 0; e < 16; ++e)
      if (!std::isfinite(corr[16 * k + e])) return fail(ctx, DCG_ERR_ARG, "correction not finite");
  }
  if (n_transformed) *n_transformed = 0;
  if (n_moved) *n_moved = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int C = (int)ctx->chunks.size();
  if (C == 0) return DCG_OK;
  // 1. frustum cull of every affected keyframe (pose before the correction)
  std::memcpy(ctx->h_cullcams, kf, sizeof(dcg_camera) * K);
  CK(cudaMemcpyAsync(ctx->d_cullcams, ctx->h_cullcams, sizeof(dcg_camera) * K, cudaMemcpyHostToDevice, s));
  hook(ctx)(PH_LOOP, true, s);
  CK(launch_cull(ctx->d_coords, C, ctx->d_cullcams, nullptr, K, ctx->cfg.chunk_size, ctx->cfg.dfar, ctx->d_lcmask,
                 ctx->d_vis, ctx->d_list, ctx->d_nlist, s));
  hook(ctx)(PH_LOOP, false, s);
  int32_t nl = 0;
  CK(cudaMemcpyAsync(&nl, ctx->d_nlist, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int32_t> list((size_t)nl);
  if (nl) CK(cudaMemcpy(list.data(), ctx->d_list, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost));
  if (nl == 0) return DCG_OK;
  // the keyframes: pose before the correction, intrinsics, correction and its rotation
  std::vector<LcView> views((size_t)K);
  for (int k = 0; k < K; ++k) {
    const dcg_camera& c = kf[k];
    LcView& v = views[(size_t)k];
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) v.R[3 * r + q] = c.Tcw[4 * r + q];
      v.t[r] = c.Tcw[4 * r + 3];
      for (int q = 0; q < 4; ++q) v.C[4 * r + q] = corr[16 * k + 4 * r + q];
    }
    v.fx = c.fx; v.fy = c.fy; v.cx = c.cx; v.cy = c.cy; v.znear = c.znear; v.zfar = c.zfar; v.W = c.W; v.H = c.H;
    double Rd[9], qd[4];
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) Rd[3 * r + q] = corr[16 * k + 4 * r + q];
    rot_to_quat(Rd, qd);
    for (int q = 0; q < 4; ++q) v.q[q] = (float)qd[q];
  }
  CK(cudaMemcpyAsync(ctx->d_lcview, views.data(), sizeof(LcView) * K, cudaMemcpyHostToDevice, s));
  // a deferred write-back goes to the pages first, as the transform works in place
  {
    dcg_status wb = writeback_active(ctx, s);
    if (wb != DCG_OK) return wb;
  }
  // 2. batch-load the union; when it exceeds the device budget, one keyframe at a time
  {
    int64_t total = 0;
    for (int k = 0; k < nl; ++k) total += ctx->chunks[(size_t)list[(size_t)k]].count;
    if (total > std::min<int64_t>(ctx->cfg.device_budget, ctx->cfg.max_active)) {
      std::vector<uint8_t> hmask((size_t)K * C);
      CK(cudaMemcpy(hmask.data(), ctx->d_lcmask, (size_t)K * C, cudaMemcpyDeviceToHost));
      return loop_closure_by_keyframe(ctx, hmask.data(), K, C, n_transformed, n_moved, s);
    }
  }
  dcg_gaussians g{};
  int64_t n = 0;
  dcg_status gs = dcg_gather_active(ctx, list.data(), nl, &g, &n, stream);
  if (gs != DCG_OK) return gs;
  std::vector<long long> seg((size_t)nl);
  std::vector<int> segc((size_t)nl);
  std::vector<uint64_t> segkey((size_t)nl);
  {
    long long off = 0;
    for (int k = 0; k < nl; ++k) {
      seg[(size_t)k] = off;
      segc[(size_t)k] = list[(size_t)k];
      segkey[(size_t)k] = ctx->chunks[list[(size_t)k]].key;
      off += ctx->chunks[list[(size_t)k]].count;
    }
  }
  CK(cudaMemcpyAsync(ctx->d_lcseg, seg.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->d_lcsegc, segc.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
  // 3. rigid correction under the global mask, then chunk ids of the result (Eq. 5/6)
  dcg_render_state* st = ctx->st0;
  uint32_t* d_flags = st->touched;  // render scratch, at least max_active entries
  u64* d_keys = st->list_a;
  const int64_t S = ctx->cfg.max_active;
  hook(ctx)(PH_LOOP, true, s);
  launch_loop_transform(ctx->d_active, S, n, ctx->d_lcseg, ctx->d_lcsegc, nl, ctx->d_lcmask, C, ctx->d_lcview, K,
                        d_flags, 0, ctx->num_sms, s);
  launch_chunk_keys(ctx->d_active, 1, S, n, ctx->cfg.chunk_size, d_keys, ctx->d_errword, ctx->num_sms, s);
  hook(ctx)(PH_LOOP, false, s);
  CK(cudaGetLastError());
  // 4. redistribution: a chunk keeps its remaining Gaussians in stored order
  // and receives incoming ones after them, in gather order.  The device marks
  // and compacts the moved rows (a rigid correction moves few across chunk
  // borders), the host plans only those and the per-chunk offsets, and the
  // device writes the permutation.
  const int Fs = ctx->Fs;
  {
    dcg_status rs = lc_reserve(ctx, n, s);
    if (rs != DCG_OK) return rs;
  }
  CK(cudaMemcpyAsync(ctx->d_lcsegkey, segkey.data(), sizeof(u64) * (size_t)nl, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ctx->d_lccnt, 0, 2 * sizeof(u64), s));
  hook(ctx)(PH_LOOP, true, s);
  launch_lc_moved(d_flags, d_keys, n, ctx->d_lcseg, ctx->d_lcsegkey, nl, (unsigned long long*)ctx->d_lccnt,
                  ctx->d_lcmidx, ctx->d_lcmkey, st->part, st->P, ctx->d_lccnt + 1, ctx->num_sms, s);
  hook(ctx)(PH_LOOP, false, s);
  CK(cudaGetLastError());
  u64 cnt[2] = {0, 0};
  CK(cudaMemcpyAsync(cnt, ctx->d_lccnt, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  dcg_status es = dcg_sync(ctx, stream);  // a corrected position outside the key range stops here, table unchanged
  if (es != DCG_OK) {
    ctx->active_valid = false;
    return es;
  }
  const int64_t nt = (int64_t)cnt[0], nm = (int64_t)cnt[1];
  if (n_transformed) *n_transformed = nt;
  if (n_moved) *n_moved = nm;
  if (nm == 0) return dcg_scatter_back(ctx, &g, n, stream);
  std::vector<long long> midx((size_t)nm);
  std::vector<uint64_t> mkey((size_t)nm);
  CK(cudaMemcpyAsync(midx.data(), ctx->d_lcmidx, sizeof(long long) * (size_t)nm, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(mkey.data(), ctx->d_lcmkey, sizeof(u64) * (size_t)nm, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // per segment: rows moving out and moved rows before its first row
  std::vector<int64_t> out_k((size_t)nl, 0), mb_k((size_t)nl, 0), size_k((size_t)nl);
  {
    int64_t m = 0;
    for (int k = 0; k < nl; ++k) {
      const int64_t end = k + 1 < nl ? seg[(size_t)k + 1] : n;
      size_k[(size_t)k] = end - seg[(size_t)k];
      mb_k[(size_t)k] = m;
      while (m < nm && midx[(size_t)m] < end) {
        ++out_k[(size_t)k];
        ++m;
      }
    }
  }
  // moved rows by target chunk, gather order kept within each
  std::vector<int64_t> order((size_t)nm);
  for (int64_t t = 0; t < nm; ++t) order[(size_t)t] = t;
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return mkey[(size_t)x] < mkey[(size_t)y]; });
  std::vector<std::pair<uint64_t, int>> keyk((size_t)nl);
  for (int k = 0; k < nl; ++k) keyk[(size_t)k] = {segkey[(size_t)k], k};
  std::sort(keyk.begin(), keyk.end());
  auto gathered = [&](uint64_t key) {  // list position of the gathered chunk with this id, or -1
    auto it = std::lower_bound(keyk.begin(), keyk.end(), std::make_pair(key, -1));
    return it != keyk.end() && it->first == key ? it->second : -1;
  };
  std::vector<int64_t> in_k((size_t)nl, 0);
  for (int64_t t = 0; t < nm; ++t) {
    const int k = gathered(mkey[(size_t)order[(size_t)t]]);
    if (k >= 0) ++in_k[(size_t)k];
  }
  std::vector<int64_t> newcount((size_t)nl), newoff((size_t)nl);
  int64_t n_kept = 0;  // Gaussians staying on the device (gathered chunks)
  for (int k = 0; k < nl; ++k) {
    newcount[(size_t)k] = size_k[(size_t)k] - out_k[(size_t)k] + in_k[(size_t)k];
    newoff[(size_t)k] = n_kept;
    n_kept += newcount[(size_t)k];
  }
  std::vector<long long> mdest((size_t)nm), base((size_t)nl);
  std::vector<int64_t> fill((size_t)nl, 0);
  std::vector<std::pair<uint64_t, int64_t>> outside;  // (key, count) of targets that were not gathered, ascending
  int64_t od = n_kept;
  for (int64_t t = 0; t < nm; ++t) {
    const int64_t pos = order[(size_t)t];
    const uint64_t key = mkey[(size_t)pos];
    const int k = gathered(key);
    if (k >= 0) {
      mdest[(size_t)pos] = newoff[(size_t)k] + size_k[(size_t)k] - out_k[(size_t)k] + fill[(size_t)k]++;
    } else {
      mdest[(size_t)pos] = od++;
      if (outside.empty() || outside.back().first != key) outside.emplace_back(key, 0);
      ++outside.back().second;
    }
  }
  for (int k = 0; k < nl; ++k) base[(size_t)k] = newoff[(size_t)k] - seg[(size_t)k] + mb_k[(size_t)k];
  // capacity checks before anything changes
  int64_t dev_need = 0, dev_have = 0, host_need = 0, host_have = 0, new_chunks = 0;
  for (int k = 0; k < nl; ++k) {
    const Chunk& ch = ctx->chunks[list[(size_t)k]];
    dev_need += pages_for(ctx, newcount[(size_t)k]);
    dev_have += (int64_t)ch.dev_pages.size();
    host_need += pages_for(ctx, newcount[(size_t)k]);
    host_have += (int64_t)ch.host_pages.size();
  }
  for (auto& o : outside) {
    auto it = ctx->index.find(o.first);
    if (it == ctx->index.end()) {
      ++new_chunks;
      host_need += pages_for(ctx, o.second);
    } else {
      const Chunk& ch = ctx->chunks[it->second];
      host_need += pages_for(ctx, ch.count + o.second) - (int64_t)ch.host_pages.size();
    }
  }
  if (dev_need - dev_have > (int64_t)ctx->dev_free.size()) return fail(ctx, DCG_ERR_BUDGET, "device page pool exhausted");
  if (host_need - host_have > (int64_t)ctx->host_free.size()) return fail(ctx, DCG_ERR_CAPACITY, "host tier full");
  if ((int64_t)ctx->chunks.size() + new_chunks > ctx->cfg.max_chunks)
    return fail(ctx, DCG_ERR_CAPACITY, "chunk table full");
  // the permutation from the planned destinations, then the permuted copy of
  // the active rows (parameters and moments)
  float* const d_tmp = ctx->d_lctmp;
  long long* const d_perm = ctx->d_lcperm;
  CK(cudaMemcpyAsync(ctx->d_lcmkey, mdest.data(), sizeof(long long) * (size_t)nm, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->d_lcsegbase, base.data(), sizeof(long long) * (size_t)nl, cudaMemcpyHostToDevice, s));
  hook(ctx)(PH_LOOP, true, s);
  launch_lc_dest(d_flags, n, ctx->d_lcseg, ctx->d_lcsegbase, nl, ctx->d_lcmidx,
                 reinterpret_cast<const long long*>(ctx->d_lcmkey), nm, d_perm, ctx->num_sms, s);
  hook(ctx)(PH_LOOP, false, s);
  hook(ctx)(PH_LOOP, true, s);
  launch_permute_rows(ctx->d_active, S, d_tmp, n, d_perm, n, Fs, ctx->num_sms, s);
  hook(ctx)(PH_LOOP, false, s);
  // gathered chunks: new counts and pages, content written from the permuted rows
  long long* hd = nullptr;
  {
    dcg_status ds = desc_stage(ctx, &hd);
    if (ds != DCG_OK) return ds;
  }
  int nd = 0;
  int64_t off = 0;
  for (int k = 0; k < nl; ++k) {
    Chunk& ch = ctx->chunks[list[(size_t)k]];
    const int64_t nc = newcount[(size_t)k];
    const size_t np = (size_t)pages_for(ctx, nc);
    while (ch.dev_pages.size() < np) {
      ch.dev_pages.push_back(ctx->dev_free.back());
      ctx->dev_free.pop_back();
    }
    while (ch.dev_pages.size() > np) {
      ctx->dev_free.push_back(ch.dev_pages.back());
      ch.dev_pages.pop_back();
    }
    while (ch.host_pages.size() < np) {
      ch.host_pages.push_back(ctx->host_free.back());
      ctx->host_free.pop_back();
    }
    while (ch.host_pages.size() > np) {
      ctx->host_free.push_back(ch.host_pages.back());
      ch.host_pages.pop_back();
    }
    ctx->resident_g += nc - ch.count;
    ch.count = nc;
    ch.dirty = true;
    for (size_t p = 0; p < np; ++p) {
      const int64_t cnt = std::min<int64_t>(ctx->page_g, nc - (int64_t)p * ctx->page_g);
      hd[3 * nd + 0] = ch.dev_pages[p];
      hd[3 * nd + 1] = cnt;
      hd[3 * nd + 2] = off;
      off += cnt;
      ++nd;
    }
  }
  {
    dcg_status us = desc_upload(ctx, nd, s);
    if (us != DCG_OK) return us;
  }
  hook(ctx)(PH_LOOP, true, s);
  launch_page_copy(false, ctx->d_pool, ctx->page_g, Fs, 0, Fs, active_desc(ctx), nd, d_tmp, n, s);
  hook(ctx)(PH_LOOP, false, s);
  CK(cudaGetLastError());
  // Gaussians leaving for chunks that were not gathered: appended in the host tier
  const int64_t n_out = n - n_kept;
  if (n_out > 0) {
    if (n_out * Fs > ctx->stage_cap) {
      if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
      ctx->h_stage = nullptr;
      ctx->stage_cap = 0;
      CK(cudaHostAlloc((void**)&ctx->h_stage, sizeof(float) * (size_t)(n_out * Fs), 0));
      ctx->stage_cap = n_out * Fs;
    }
    CK(cudaMemcpy2DAsync(ctx->h_stage, (size_t)n_out * 4, d_tmp + n_kept, (size_t)n * 4, (size_t)n_out * 4, (size_t)Fs,
                         cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  if (n_out > 0) {
    bool added = false;
    int64_t j = 0;
    for (auto& o : outside) {
      auto it = ctx->index.find(o.first);
      if (it == ctx->index.end()) {
        ctx->chunks.push_back(make_chunk(o.first));
        ctx->index[o.first] = (int32_t)ctx->chunks.size() - 1;
        added = true;
        it = ctx->index.find(o.first);
      }
      Chunk& ch = ctx->chunks[it->second];
      if (ch.resident) {  // write back and drop: the next gather reloads the whole chunk
        CK(cudaEventRecord(ctx->ev_compute, s));
        CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_compute, 0));
        dcg_status e = evict_chunk(ctx, ch);
        if (e != DCG_OK) return e;
        ctx->evictions--;
        CK(cudaStreamSynchronize(ctx->copy_stream));
      }
      for (int64_t q = 0; q < o.second; ++q, ++j) append_host_row(ctx, ch, ctx->h_stage, n_out, j, Fs);
    }
    if (added) {
      std::sort(ctx->chunks.begin(), ctx->chunks.end(), [](const Chunk& a, const Chunk& b) { return a.key < b.key; });
      ctx->index.clear();
      for (size_t k = 0; k < ctx->chunks.size(); ++k) ctx->index[ctx->chunks[k].key] = (int32_t)k;
      dcg_status us = upload_coords(ctx);
      if (us != DCG_OK) return us;
    }
  }
  ctx->active_valid = false;  // the caller gathers again
  ctx->active_fresh = false;
  ctx->active_dirty = false;
  return DCG_OK;
}

dcg_status dcg_reset_active(dcg_ctx* ctx, const dcg_gaussians* params, int64_t n, float max_opacity, void* stream) {
  if (!ctx || !params || !params->data || !(max_opacity > 0.f && max_opacity < 1.f))
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if (!ctx->active_valid || n != ctx->n_active) return fail(ctx, DCG_ERR_STATE, "n must equal the gathered active set");
  if (params->sh_degree != ctx->cfg.sh_degree || params->stride < n) return fail(ctx, DCG_ERR_ARG, "bad layout");
  cudaStream_t s = (cudaStream_t)stream;
  const float cap = (float)std::log((double)max_opacity / (1.0 - (double)max_opacity));
  launch_cap_rows(params->data + 10 * params->stride, n, cap, ctx->num_sms, s);
  if (ctx->Fs > ctx->F)
    CK(cudaMemset2DAsync(ctx->d_active + (size_t)ctx->F * ctx->cfg.max_active, (size_t)ctx->cfg.max_active * 4, 0,
                         (size_t)n * 4, (size_t)(ctx->Fs - ctx->F), s));
  CK(cudaGetLastError());
  return DCG_OK;
}

// ---------------------------------------------------------------- LoG sampling
static LcView view_of(const dcg_camera& c) {
  LcView v{};
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) v.R[3 * r + q] = c.Tcw[4 * r + q];
    v.t[r] = c.Tcw[4 * r + 3];
  }
  v.fx = c.fx; v.fy = c.fy; v.cx = c.cx; v.cy = c.cy; v.znear = c.znear; v.zfar = c.zfar; v.W = c.W; v.H = c.H;
  return v;
}

static_assert(kLsMaxViews == kMaxViewsApi, "one view limit for the sampling calls and the rest of the ABI");

// Table of the views of one sampling / back-projection call: window offsets
// and penalty tiles.  False if a view is empty or the window is too large.
static bool ls_table(const dcg_camera* cams, int V, bool with_pose, LsViews* t) {
  *t = LsViews{};
  t->V = V;
  long long off = 0;
  int tiles = 0;
  for (int v = 0; v < V; ++v) {
    const dcg_camera& c = cams[v];
    if (c.W <= 0 || c.H <= 0) return false;
    if (with_pose && (!(c.fx > 0.f) || !(c.fy > 0.f))) return false;
    LsView& w = t->v[v];
    if (with_pose) {
      w.cam = view_of(c);
    } else {
      w.cam.W = c.W;
      w.cam.H = c.H;
    }
    w.off = off;
    w.tile0 = tiles;
    w.ntx = (c.W + kLsTile - 1) / kLsTile;
    const long long nt = (long long)w.ntx * ((c.H + kLsTile - 1) / kLsTile);
    off += (long long)c.W * c.H;
    if (off >= (1ll << 31) || tiles + nt >= (1ll << 31)) return false;
    tiles += (int)nt;
  }
  t->n_tiles = tiles;
  t->n_pix = off;
  return true;
}

static dcg_status log_sample_run(dcg_ctx* ctx, const LsViews& t, const float* image, const float* rendered, float kappa,
                                 const float* u, float* ps_out, int32_t* idx_out, int64_t max_out, int64_t* counts,
                                 int64_t* n_out, cudaStream_t s) {
  if (t.n_pix > ctx->cfg.max_pixels) return fail(ctx, DCG_ERR_CAPACITY, "more pixels than max_pixels");
  dcg_render_state* st = ctx->st0;
  hook(ctx)(PH_SAMPLE, true, s);
  launch_log_sample(image, rendered, t, kappa, u, ps_out, ctx->d_lsflags, idx_out, max_out, st->part, st->P,
                    ctx->d_lscount, ctx->d_lsvcount, s);
  hook(ctx)(PH_SAMPLE, false, s);
  CK(cudaGetLastError());
  u64 cnt = 0;
  u64 vc[kLsMaxViews] = {};
  CK(cudaMemcpyAsync(&cnt, ctx->d_lscount, sizeof(u64), cudaMemcpyDeviceToHost, s));
  if (counts) CK(cudaMemcpyAsync(vc, ctx->d_lsvcount, sizeof(u64) * t.V, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *n_out = (int64_t)std::min<u64>(cnt, (u64)max_out);
  if (counts)
    for (int v = 0; v < t.V; ++v) counts[v] = (int64_t)vc[v];
  if (cnt > (u64)max_out) return fail(ctx, DCG_ERR_CAPACITY, "more samples than max_out");
  return DCG_OK;
}

dcg_status dcg_log_sample(dcg_ctx* ctx, const float* image, const float* rendered, int32_t W, int32_t H, float kappa,
                          const float* u, float* ps_out, int32_t* idx_out, int32_t max_out, int32_t* n_out,
                          void* stream) {
  if (!ctx || !image || !rendered || !u || !idx_out || !n_out || W <= 0 || H <= 0 || max_out < 0 || !(kappa >= 0.f) ||
      !std::isfinite(kappa))
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if ((int64_t)W * H > ctx->cfg.max_pixels || (int64_t)W * H >= (1ll << 31))
    return fail(ctx, DCG_ERR_CAPACITY, "image larger than max_pixels");
  dcg_camera c{};
  c.W = W;
  c.H = H;
  LsViews t;
  ls_table(&c, 1, false, &t);
  int64_t n = 0;
  const dcg_status r = log_sample_run(ctx, t, image, rendered, kappa, u, ps_out, idx_out, max_out, nullptr, &n,
                                      (cudaStream_t)stream);
  *n_out = (int32_t)n;
  return r;
}

dcg_status dcg_log_sample_views(dcg_ctx* ctx, const dcg_camera* cams, int32_t n_views, const float* image,
                                const float* rendered, float kappa, const float* u, float* ps_out, int32_t* idx_out,
                                int64_t max_out, int64_t* counts, int64_t* n_out, void* stream) {
  if (!ctx || !cams || n_views <= 0 || n_views > kLsMaxViews || !image || !rendered || !u || !idx_out || !n_out ||
      max_out < 0 || !(kappa >= 0.f) || !std::isfinite(kappa))
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  LsViews t;
  if (!ls_table(cams, n_views, false, &t)) return fail(ctx, DCG_ERR_ARG, "empty view or window of 2^31 pixels or more");
  return log_sample_run(ctx, t, image, rendered, kappa, u, ps_out, idx_out, max_out, counts, n_out,
                        (cudaStream_t)stream);
}

static dcg_status backproject_run(dcg_ctx* ctx, const LsViews& t, const int32_t* idx, int64_t n, const float* depth,
                                  const float* image, float opacity_logit, float* params_out, int64_t stride,
                                  cudaStream_t s) {
  hook(ctx)(PH_SAMPLE, true, s);
  launch_backproject(idx, n, depth, image, t, opacity_logit, ctx->F, params_out, stride, ctx->num_sms, s);
  hook(ctx)(PH_SAMPLE, false, s);
  CK(cudaGetLastError());
  return DCG_OK;
}

dcg_status dcg_backproject(dcg_ctx* ctx, const int32_t* idx, int32_t n, const float* depth, const float* image,
                           const dcg_camera* cam, float opacity_logit, float* params_out, int64_t stride,
                           void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!idx || !depth || !image || !params_out)) || !cam || stride < n)
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  LsViews t;
  if (!ls_table(cam, 1, true, &t)) return fail(ctx, DCG_ERR_ARG, "bad camera");
  return backproject_run(ctx, t, idx, n, depth, image, opacity_logit, params_out, stride, (cudaStream_t)stream);
}

dcg_status dcg_backproject_views(dcg_ctx* ctx, const int32_t* idx, int64_t n, const float* depth, const float* image,
                                 const dcg_camera* cams, int32_t n_views, float opacity_logit, float* params_out,
                                 int64_t stride, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!idx || !depth || !image || !params_out)) || !cams || n_views <= 0 ||
      n_views > kLsMaxViews || stride < n)
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  LsViews t;
  if (!ls_table(cams, n_views, true, &t)) return fail(ctx, DCG_ERR_ARG, "bad camera or window of 2^31 pixels or more");
  return backproject_run(ctx, t, idx, n, depth, image, opacity_logit, params_out, stride, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- rendering
dcg_status dcg_state_create(dcg_ctx* ctx, dcg_render_state** out) {
  if (!ctx || !out) return DCG_ERR_ARG;
  dcg_render_state* st = new dcg_render_state();
  dcg_status s = state_alloc(ctx, st);
  if (s != DCG_OK) {
    state_free(st);
    delete st;
    return s;
  }
  *out = st;
  return DCG_OK;
}

dcg_render_state* dcg_default_state(dcg_ctx* ctx) { return ctx ? ctx->st0 : nullptr; }

dcg_status dcg_state_destroy(dcg_render_state* st) {
  if (!st) return DCG_ERR_ARG;
  cudaDeviceSynchronize();
  state_free(st);
  delete st;
  return DCG_OK;
}

dcg_status dcg_set_launch(dcg_ctx* ctx, int32_t tw, int32_t th, int32_t stage) {
  if (!ctx || !valid_tile(tw, th) || !valid_stage(stage))
    return fail(ctx, DCG_ERR_ARG, "bad launch shape");
  ctx->tile_w = tw;
  ctx->tile_h = th;
  ctx->stage = stage;
  return DCG_OK;
}

static void fill_args(dcg_render_state* st, RasterArgs& a) {
  dcg_ctx* ctx = st->ctx;
  a.g = st->g.data;
  a.stride = st->g.stride;
  a.n = st->n;
  a.deg = st->g.sh_degree;
  a.V = st->V;
  a.cams = st->d_cams;
  a.tile_w = st->tile_w;
  a.tile_h = st->tile_h;
  a.stage = st->stage;
  a.n_tiles = st->n_tiles;
  a.n_pix = st->n_pix;
  a.idx_bits = st->idx_bits;
  a.view_bits = st->view_bits;
  a.rec = st->rec;
  a.depth = st->depth;
  a.touched = st->touched;
  a.rect = st->rect;
  a.bin = st->bin;
  a.grad2d = st->grad2d;
  a.list_a = st->list_a;
  a.list_b = st->list_b;
  a.inst_a = st->inst_a;
  a.inst_b = st->inst_b;
  a.cap_pairs = st->cap_pairs;
  a.cap_inst = st->cap_inst;
  a.ranges = st->ranges;
  a.T_final = st->T_final;
  a.n_contrib = st->n_contrib;
  a.counters = st->counters;
  a.part = st->part;
  a.hist = st->hist;
  a.P = st->P;
  a.errword = ctx->d_errword;
  a.num_sms = ctx->num_sms;
  a.prof = hook(ctx);
  a.bwd_slots = (ctx->cfg.flags & 1) ? 1 : 0;
  a.bwd_pix = (ctx->cfg.flags & 2) ? 1 : 0;
}

static void fill_devcams(const dcg_camera* cams, int V, int tw, int th, DevCam* out, int64_t* pix_out,
                         int* tiles_out) {
  int64_t pix = 0;
  int tiles = 0;
  for (int v = 0; v < V; ++v) {
    const dcg_camera& c = cams[v];
    DevCam& d = out[v];
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) d.R[3 * r + k] = c.Tcw[4 * r + k];
      d.t[r] = c.Tcw[4 * r + 3];
    }
    for (int k = 0; k < 3; ++k)
      d.C[k] = (float)(-((double)c.Tcw[0 + k] * c.Tcw[3] + (double)c.Tcw[4 + k] * c.Tcw[7] + (double)c.Tcw[8 + k] * c.Tcw[11]));
    d.znear = c.znear; d.zfar = c.zfar;
    d.xlo = (float)((-0.15 * c.W - c.cx) / c.fx);
    d.xhi = (float)((1.15 * c.W - c.cx) / c.fx);
    d.ylo = (float)((-0.15 * c.H - c.cy) / c.fy);
    d.yhi = (float)((1.15 * c.H - c.cy) / c.fy);
    d.W = c.W; d.H = c.H;
    d.ntx = (c.W + tw - 1) / tw;
    d.nty = (c.H + th - 1) / th;
    d.tile_base = tiles;
    d.pad = 0;
    d.pix_off = pix;
    tiles += d.ntx * d.nty;
    pix += (int64_t)c.W * c.H;
  }
  *pix_out = pix;
  *tiles_out = tiles;
}

dcg_status dcg_render_fwd(dcg_ctx* ctx, const dcg_gaussians* g, int64_t n, const dcg_camera* cams, int32_t V,
                          float* rgb, float* depth, dcg_render_state* st, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  if (!st) st = ctx->st0;
  if (!g || n < 0 || (n > 0 && !g->data) || g->stride < n || g->sh_degree < 0 || g->sh_degree > 3 || !rgb || !depth)
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  dcg_status cs = check_cams(ctx, cams, V);
  if (cs != DCG_OK) return cs;
  if (n > st->cap_n) return fail(ctx, DCG_ERR_CAPACITY, "more Gaussians than max_active");
  cudaStream_t s = (cudaStream_t)stream;
  const int tw = ctx->tile_w, th = ctx->tile_h;
  int64_t pix = 0;
  int tiles = 0;
  CK(cudaEventSynchronize(st->ev_cams));  // staging buffer free again
  fill_devcams(cams, V, tw, th, st->h_cams, &pix, &tiles);
  if (pix > st->cap_pix || tiles > st->cap_tiles || tiles > kMaxTiles)
    return fail(ctx, DCG_ERR_CAPACITY, "pixel or tile capacity exceeded");
  CK(cudaMemcpyAsync(st->d_cams, st->h_cams, sizeof(DevCam) * V, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(st->ev_cams, s));
  st->g = *g;
  st->n = n;
  st->V = V;
  st->n_pix = pix;
  st->n_tiles = tiles;
  st->tile_w = tw;
  st->tile_h = th;
  st->stage = ctx->stage;
  st->idx_bits = 1;
  while ((1ll << st->idx_bits) < n) ++st->idx_bits;
  st->view_bits = 0;
  while ((1 << st->view_bits) < V) ++st->view_bits;
  RasterArgs a;
  fill_args(st, a);
  raster_forward(a, rgb, depth, &st->list_sorted, &st->inst_sorted, s);
  CK(cudaGetLastError());
  st->valid = true;
  st->gen++;
  return DCG_OK;
}

dcg_status dcg_render_bwd(dcg_ctx* ctx, dcg_render_state* st, const float* dL_drgb, const float* dL_ddepth,
                          dcg_gaussians* grads, float* dL_dpose, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  if (!st) st = ctx->st0;
  if (!st->valid) return fail(ctx, DCG_ERR_STATE, "backward without a forward");
  if (!dL_drgb || !dL_ddepth || !grads || (st->n > 0 && !grads->data) || grads->stride < st->n ||
      grads->sh_degree != st->g.sh_degree)
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  RasterArgs a;
  fill_args(st, a);
  raster_backward(a, st->inst_sorted, dL_drgb, dL_ddepth, grads->data, grads->stride, dL_dpose, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return DCG_OK;
}

// 16 x 16 tiles of the views for the SSIM kernel; returns the tile count.
static int64_t fill_ssim_cams(const dcg_camera* cams, int V, DevCam* out) {
  const int t = ssim_tile();
  int64_t pix = 0, tiles = 0;
  for (int v = 0; v < V; ++v) {
    DevCam& d = out[v];
    std::memset(&d, 0, sizeof(d));
    d.W = cams[v].W;
    d.H = cams[v].H;
    d.pix_off = pix;
    d.ntx = (d.W + t - 1) / t;
    d.nty = (d.H + t - 1) / t;
    d.tile_base = (int)tiles;
    pix += (int64_t)d.W * d.H;
    tiles += (int64_t)d.ntx * d.nty;
  }
  return tiles;
}

static dcg_status loss_impl(dcg_ctx* ctx, const float* rgb, const float* depth, const float* trgb, const float* tdepth,
                            const dcg_camera* cams, int32_t V, float lambda_s, float lam, float* dr, float* dd,
                            float* loss, void* stream) {
  if (!ctx || !rgb || !depth || !trgb || !tdepth || !dr || !dd || !loss) return fail(ctx, DCG_ERR_ARG, "bad arguments");
  if (!(lambda_s >= 0.f && lambda_s <= 1.f) || !std::isfinite(lam)) return fail(ctx, DCG_ERR_ARG, "bad loss weights");
  dcg_status cs = check_cams(ctx, cams, V);
  if (cs != DCG_OK) return cs;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaEventSynchronize(ctx->ev_loss));  // staging buffers free again
  int64_t pix = 0;
  for (int v = 0; v < V; ++v) {
    DevCam& d = ctx->h_losscams[v];
    std::memset(&d, 0, sizeof(d));
    d.W = cams[v].W;
    d.H = cams[v].H;
    d.pix_off = pix;
    pix += (int64_t)cams[v].W * cams[v].H;
  }
  const int64_t tiles = lambda_s > 0.f ? fill_ssim_cams(cams, V, ctx->h_ssimcams) : 0;
  if (tiles > ctx->cap_ssim_tiles) return fail(ctx, DCG_ERR_CAPACITY, "SSIM tile capacity exceeded");
  CK(cudaMemcpyAsync(ctx->d_losscams, ctx->h_losscams, sizeof(DevCam) * V, cudaMemcpyHostToDevice, s));
  if (tiles) CK(cudaMemcpyAsync(ctx->d_ssimcams, ctx->h_ssimcams, sizeof(DevCam) * V, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(ctx->ev_loss, s));
  hook(ctx)(PH_LOSS, true, s);
  launch_loss_l1(rgb, depth, trgb, tdepth, ctx->d_losscams, V, pix, 1.f - lambda_s, lam, dr, dd, loss,
                 ctx->d_losspart, ctx->num_sms, s);
  if (tiles) launch_ssim(rgb, trgb, ctx->d_ssimcams, V, (int)tiles, lambda_s, dr, loss, ctx->d_ssimpart, s);
  hook(ctx)(PH_LOSS, false, s);
  CK(cudaGetLastError());
  return DCG_OK;
}

dcg_status dcg_loss_l1(dcg_ctx* ctx, const float* rgb, const float* depth, const float* trgb, const float* tdepth,
                       const dcg_camera* cams, int32_t V, float lam, float* dr, float* dd, float* loss, void* stream) {
  return loss_impl(ctx, rgb, depth, trgb, tdepth, cams, V, 0.f, lam, dr, dd, loss, stream);
}

dcg_status dcg_loss(dcg_ctx* ctx, const float* rgb, const float* depth, const float* trgb, const float* tdepth,
                    const dcg_camera* cams, int32_t V, float lambda_s, float lambda_depth, float* dr, float* dd,
                    float* loss, void* stream) {
  return loss_impl(ctx, rgb, depth, trgb, tdepth, cams, V, lambda_s, lambda_depth, dr, dd, loss, stream);
}

dcg_status dcg_window_capture(dcg_ctx* ctx, const dcg_gaussians* g, int64_t n, const dcg_camera* cams, int32_t V,
                              float* rgb, float* depth, const float* trgb, const float* tdepth, float lam,
                              float lambda_s, float* dr, float* dd, float* loss, dcg_gaussians* grads, float* dL_dpose,
                              void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  dcg_render_state* st = ctx->st0;
  if (!g || n < 0 || (n > 0 && !g->data) || g->stride < n || !rgb || !depth || !trgb || !tdepth || !dr || !dd ||
      !loss || !grads || grads->stride < n || grads->sh_degree != g->sh_degree || !(lambda_s >= 0.f && lambda_s <= 1.f))
    return fail(ctx, DCG_ERR_ARG, "bad arguments");
  dcg_status cs = check_cams(ctx, cams, V);
  if (cs != DCG_OK) return cs;
  if (n > st->cap_n) return fail(ctx, DCG_ERR_CAPACITY, "more Gaussians than max_active");
  cudaStream_t s = (cudaStream_t)stream;
  const int tw = ctx->tile_w, th = ctx->tile_h;
  CK(cudaStreamSynchronize(s));
  int64_t pix = 0;
  int tiles = 0;
  fill_devcams(cams, V, tw, th, ctx->h_wcams, &pix, &tiles);
  if (pix > st->cap_pix || tiles > st->cap_tiles || tiles > kMaxTiles)
    return fail(ctx, DCG_ERR_CAPACITY, "pixel or tile capacity exceeded");
  // loss cameras (pixel offsets) live in the second half of the staging buffer
  DevCam* lc = ctx->h_wcams + kMaxViewsApi;
  for (int v = 0; v < V; ++v) lc[v] = ctx->h_wcams[v];
  DevCam* sc = ctx->h_ssimcams + kMaxViewsApi;
  const int64_t stiles = lambda_s > 0.f ? fill_ssim_cams(cams, V, sc) : 0;
  if (stiles > ctx->cap_ssim_tiles) return fail(ctx, DCG_ERR_CAPACITY, "SSIM tile capacity exceeded");
  st->g = *g;
  st->n = n;
  st->V = V;
  st->n_pix = pix;
  st->n_tiles = tiles;
  st->tile_w = tw;
  st->tile_h = th;
  st->stage = ctx->stage;
  st->idx_bits = 1;
  while ((1ll << st->idx_bits) < n) ++st->idx_bits;
  st->view_bits = 0;
  while ((1 << st->view_bits) < V) ++st->view_bits;
  RasterArgs a;
  fill_args(st, a);
  a.prof = ProfHook();
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;
  const unsigned long long l0 = g_launches;
  cudaGraph_t graph = nullptr;
  cudaStream_t cs_ = ctx->cap_stream;
  const cudaError_t be = cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal);
  if (be != cudaSuccess) {
    ctx->prof_on = prof;
    cudaGetLastError();
    return fail(ctx, DCG_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(be));
  }
  cudaMemcpyAsync(st->d_cams, ctx->h_wcams, sizeof(DevCam) * V, cudaMemcpyHostToDevice, cs_);
  cudaMemcpyAsync(ctx->d_losscams, lc, sizeof(DevCam) * V, cudaMemcpyHostToDevice, cs_);
  if (stiles) cudaMemcpyAsync(ctx->d_wssimcams, sc, sizeof(DevCam) * V, cudaMemcpyHostToDevice, cs_);
  cudaMemsetAsync(loss, 0, sizeof(float), cs_);
  raster_forward(a, rgb, depth, &st->list_sorted, &st->inst_sorted, cs_);
  launch_loss_l1(rgb, depth, trgb, tdepth, ctx->d_losscams, V, pix, 1.f - lambda_s, lam, dr, dd, loss,
                 ctx->d_losspart, ctx->num_sms, cs_);
  if (stiles) launch_ssim(rgb, trgb, ctx->d_wssimcams, V, (int)stiles, lambda_s, dr, loss, ctx->d_ssimpart, cs_);
  raster_backward(a, st->inst_sorted, dr, dd, grads->data, grads->stride, dL_dpose, cs_);
  const cudaError_t ce = cudaStreamEndCapture(cs_, &graph);
  ctx->prof_on = prof;
  ctx->win_kernels = g_launches - l0;
  g_launches = l0;  // capture launches nothing; replays are counted in dcg_window_run
  if (ce != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return fail(ctx, DCG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
  }
  if (ctx->win_exec) cudaGraphExecDestroy(ctx->win_exec);
  ctx->win_exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ctx->win_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(ctx, DCG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ie));
  ctx->win_V = V;
  for (int v = 0; v < V; ++v) {
    ctx->win_W[v] = cams[v].W;
    ctx->win_H[v] = cams[v].H;
  }
  ctx->win_launch[0] = tw;
  ctx->win_launch[1] = th;
  ctx->win_launch[2] = ctx->stage;
  st->valid = true;
  st->gen++;
  CK(cudaEventRecord(ctx->ev_win, s));
  return DCG_OK;
}

dcg_status dcg_window_run(dcg_ctx* ctx, const dcg_camera* cams, int32_t V, void* stream) {
  if (!ctx) return DCG_ERR_ARG;
  if (!ctx->win_exec) return fail(ctx, DCG_ERR_STATE, "no captured window");
  dcg_status cs = check_cams(ctx, cams, V);
  if (cs != DCG_OK) return cs;
  if (V != ctx->win_V) return fail(ctx, DCG_ERR_ARG, "view count differs from the capture");
  for (int v = 0; v < V; ++v)
    if (cams[v].W != ctx->win_W[v] || cams[v].H != ctx->win_H[v])
      return fail(ctx, DCG_ERR_ARG, "image size differs from the capture");
  if (ctx->tile_w != ctx->win_launch[0] || ctx->tile_h != ctx->win_launch[1] || ctx->stage != ctx->win_launch[2])
    return fail(ctx, DCG_ERR_ARG, "launch shape changed since the capture");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaEventSynchronize(ctx->ev_win));  // the previous replay has read the camera staging
  int64_t pix = 0;
  int tiles = 0;
  fill_devcams(cams, V, ctx->win_launch[0], ctx->win_launch[1], ctx->h_wcams, &pix, &tiles);
  CK(cudaGraphLaunch(ctx->win_exec, s));
  CK(cudaEventRecord(ctx->ev_win, s));
  g_launches += ctx->win_kernels;
  ctx->st0->gen++;
  return DCG_OK;
}

int64_t dcg_state_generation(const dcg_render_state* st) { return st ? st->gen : -1; }

dcg_status dcg_autotune(dcg_ctx* ctx, const dcg_gaussians* g, int64_t n, const dcg_camera* cams, int32_t V,
                        float* rgb, float* depth, const float* dr, const float* dd, dcg_gaussians* grads, int32_t reps,
                        int32_t* tile_w, int32_t* tile_h, int32_t* stage, float* ms_out, void* stream) {
  if (!ctx || reps <= 0) return DCG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  static const int tiles[3][2] = {{16, 16}, {32, 16}, {32, 32}};
  // stage codes 32 and 16 select the warp-per-block and half-warp kernels (no staging segment)
  constexpr int NS = 7;
  static const int stages[NS] = {64, 96, 128, 192, 256, 32, 16};
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  int bt = 0, bs = 2;
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;
  dcg_status rc = DCG_OK;
  for (int t = 0; t < 3 && rc == DCG_OK; ++t)
    for (int k = 0; k < NS && rc == DCG_OK; ++k) {
      dcg_set_launch(ctx, tiles[t][0], tiles[t][1], stages[k]);
      float ms = 0.f;
      for (int r = 0; r <= reps && rc == DCG_OK; ++r) {
        if (r == 1) cudaEventRecord(a, s);
        rc = dcg_render_fwd(ctx, g, n, cams, V, rgb, depth, nullptr, stream);
        if (rc == DCG_OK) rc = dcg_render_bwd(ctx, nullptr, dr, dd, grads, nullptr, stream);
      }
      if (rc != DCG_OK) break;
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
      ms /= reps;
      if (ms_out) ms_out[NS * t + k] = ms;
      if (ms < best) {
        best = ms;
        bt = t;
        bs = k;
      }
    }
  ctx->prof_on = prof;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != DCG_OK) return rc;
  dcg_set_launch(ctx, tiles[bt][0], tiles[bt][1], stages[bs]);
  if (tile_w) *tile_w = tiles[bt][0];
  if (tile_h) *tile_h = tiles[bt][1];
  if (stage) *stage = stages[bs];
  return dcg_sync(ctx, stream);
}

dcg_status dcg_profile(dcg_ctx* ctx, int32_t enable) {
  if (!ctx) return DCG_ERR_ARG;
  if (enable && ctx->ev_pool.empty()) {
    ctx->ev_pool.resize(8192);
    for (auto& e : ctx->ev_pool) CK(cudaEventCreate(&e));
  }
  ctx->prof_on = enable != 0;
  return DCG_OK;
}

dcg_status dcg_profile_read(dcg_ctx* ctx, float* ms, int32_t* counts) {
  if (!ctx || !ms) return DCG_ERR_ARG;
  for (int p = 0; p < PH_COUNT; ++p) {
    ms[p] = 0.f;
    if (counts) counts[p] = 0;
  }
  for (auto& r : ctx->recs) {
    CK(cudaEventSynchronize(r.b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.phase] += t;
    if (counts) counts[r.phase] += 1;
  }
  ctx->recs.clear();
  ctx->ev_next = 0;
  for (auto& e : ctx->open_ev) e = nullptr;
  if (ctx->ev_dropped) {
    const uint64_t d = ctx->ev_dropped;
    ctx->ev_dropped = 0;
    return fail(ctx, DCG_ERR_CAPACITY,
                "phase timers full: " + std::to_string(d) + " marks since the last read were not recorded "
                "(the figures returned are partial; read more often)");
  }
  return DCG_OK;
}

uint64_t dcg_launch_count(void) { return (uint64_t)g_launches; }

dcg_status dcg_state_stats(dcg_render_state* st, int64_t* n_visible, int64_t* n_instances, int64_t* n_tiles,
                           void* stream) {
  if (!st) return DCG_ERR_ARG;
  DevCounters h;
  dcg_ctx* ctx = st->ctx;
  CK(cudaMemcpyAsync(&h, st->counters, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (n_visible) *n_visible = (int64_t)h.n_vis;
  if (n_instances) *n_instances = (int64_t)h.n_inst;
  if (n_tiles) *n_tiles = st->n_tiles;
  return DCG_OK;
}

dcg_status dcg_state_evals(dcg_render_state* st, int64_t* n_eval, int64_t* n_blend, void* stream) {
  if (!st || !n_eval) return DCG_ERR_ARG;
  dcg_ctx* ctx = st->ctx;
  DevCounters h;
  CK(cudaMemcpyAsync(&h, st->counters, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  *n_eval = (int64_t)h.n_eval;
  if (n_blend) *n_blend = (int64_t)h.n_blend;
  return DCG_OK;
}

dcg_status dcg_state_read(dcg_render_state* st, uint32_t* ranges, uint32_t* ids, uint16_t* masks, float* depth,
                          int32_t* rect, float* T_final, int32_t* n_contrib, void* stream) {
  if (!st || !st->valid) return DCG_ERR_STATE;
  dcg_ctx* ctx = st->ctx;
  cudaStream_t s = (cudaStream_t)stream;
  DevCounters h;
  CK(cudaMemcpyAsync(&h, st->counters, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t K = (int64_t)h.n_inst_c, pairs = (int64_t)st->V * st->n;
  if (ranges) CK(cudaMemcpyAsync(ranges, st->ranges, sizeof(uint2) * st->n_tiles, cudaMemcpyDeviceToHost, s));
  std::vector<u64> inst;
  if (ids || masks) {
    inst.resize((size_t)K);
    if (K) CK(cudaMemcpyAsync(inst.data(), st->inst_sorted, 8 * (size_t)K, cudaMemcpyDeviceToHost, s));
  }
  if (depth && pairs) CK(cudaMemcpyAsync(depth, st->depth, 4 * (size_t)pairs, cudaMemcpyDeviceToHost, s));
  std::vector<short4> r;
  if (rect) {
    r.resize((size_t)pairs);
    if (pairs) CK(cudaMemcpyAsync(r.data(), st->rect, sizeof(short4) * (size_t)pairs, cudaMemcpyDeviceToHost, s));
  }
  if (T_final) CK(cudaMemcpyAsync(T_final, st->T_final, 4 * (size_t)st->n_pix, cudaMemcpyDeviceToHost, s));
  if (n_contrib) CK(cudaMemcpyAsync(n_contrib, st->n_contrib, 4 * (size_t)st->n_pix, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (ids)
    for (int64_t k = 0; k < K; ++k) ids[k] = (uint32_t)(inst[(size_t)k] & ((1ull << 28) - 1));
  if (masks)
    for (int64_t k = 0; k < K; ++k) masks[k] = (uint16_t)(inst[(size_t)k] >> 48);
  if (rect)
    for (int64_t k = 0; k < pairs; ++k) {
      rect[4 * k + 0] = r[(size_t)k].x;
      rect[4 * k + 1] = r[(size_t)k].y;
      rect[4 * k + 2] = r[(size_t)k].z;
      rect[4 * k + 3] = r[(size_t)k].w;
    }
  return DCG_OK;
}

}  // extern "C"
