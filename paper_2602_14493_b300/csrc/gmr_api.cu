// C ABI entry points (include/gmr.h): context, workspace, argument checks and
// the order of the kernels of one forward / backward.

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gmr_internal.cuh"

using gmr::Counters;
using gmr::ViewInfo;
using gmr::Workspace;

namespace gmr {
bool chained_launch_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("GMR_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
}  // namespace gmr

struct gmr_ctx {
  gmr_config cfg;
  int device = 0;
  Workspace ws;
  std::string err;
  int64_t launches = 0;
  // cameras of the last upload
  std::vector<gmr_camera> cams;
  std::vector<ViewInfo> views;
  ViewInfo* views_pinned = nullptr;
  int32_t views_pinned_cap = 0;
  cudaEvent_t upload_done = nullptr;
  Counters* counters_pinned = nullptr;
  // stage events (GMR_FLAG_PROFILE)
  cudaEvent_t stage_ev[2 * GMR_NUM_STAGES] = {};
  uint32_t stage_mask = 0;
  // forward state consumed by the backward
  bool fwd_valid = false;
  // The last forward zeroed the record and face gradient sums and the
  // backward evaluation counter, and no backward has run since; with the
  // id of the stream capture that forward was enqueued in (0: none). A
  // backward enqueued in the same capture (or, uncaptured, after an
  // uncaptured forward) then needs no memsets of its own.
  bool grads_zero = false;
  unsigned long long grads_zero_capture = 0;
  const float* verts = nullptr;
  const int32_t* faces = nullptr;
  const float* rgb = nullptr;
  const float* opacity = nullptr;
  int32_t V = 0, F = 0, C = 0;
  int64_t n_tiles = 0, n_pixels = 0;
  int64_t n_btiles = 0;  // binning tiles of the last forward (= n_tiles unless split)
  bool split = false;    // the last forward binned 8x8 tiles as 16x16 and split the lists
  gmr_config fwd_cfg;
  // device bytes held by the workspace (per allocation, and the total), and
  // the most it may hold (0: no limit; gmr_set_workspace_limit)
  std::unordered_map<void*, size_t> dev_sizes;
  int64_t dev_bytes = 0;
  int64_t dev_limit = 0;
};

namespace {

// Workspace allocation bookkeeping (for gmr_stats.workspace_bytes).
void track_alloc(gmr_ctx* ctx, void* p, size_t bytes) {
  ctx->dev_sizes[p] = bytes;
  ctx->dev_bytes += (int64_t)bytes;
}
void track_free(gmr_ctx* ctx, void* p) {
  auto it = ctx->dev_sizes.find(p);
  if (it == ctx->dev_sizes.end()) return;
  ctx->dev_bytes -= (int64_t)it->second;
  ctx->dev_sizes.erase(it);
}

// Whether replacing the allocation `old` (may be null) by one of `bytes`
// bytes keeps the workspace within its limit.
bool within_limit(const gmr_ctx* ctx, const void* old, size_t bytes) {
  if (ctx->dev_limit <= 0) return true;
  int64_t held = ctx->dev_bytes;
  auto it = old ? ctx->dev_sizes.find(const_cast<void*>(old)) : ctx->dev_sizes.end();
  if (it != ctx->dev_sizes.end()) held -= (int64_t)it->second;
  return held + (int64_t)bytes <= ctx->dev_limit;
}

gmr_status fail(gmr_ctx* ctx, gmr_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

gmr_status cuda_fail(gmr_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, GMR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GMR_CUDA(ctx, call)                                      \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);   \
  } while (0)

bool valid_config(const gmr_config* c, std::string* why) {
  if (c->tile != 8 && c->tile != 16 && c->tile != 32) { *why = "tile must be 8, 16 or 32"; return false; }
  if (c->profile_stages >> GMR_NUM_STAGES) {
    *why = "profile_stages has bits beyond the last stage";
    return false;
  }
  for (int32_t th : {c->threads, c->threads_bwd}) {
    if (c->tile == 16 && th != 64 && th != 128 && th != 256) {
      *why = "threads must be 64, 128 or 256 with 16x16 tiles";
      return false;
    }
    if (c->tile == 32 && th != 256) { *why = "threads must be 256 with 32x32 tiles"; return false; }
    if (c->tile == 8 && th != 32 && th != 64) { *why = "threads must be 32 or 64 with 8x8 tiles"; return false; }
  }
  if (c->batch != 64 && c->batch != 128 && c->batch != 256) { *why = "batch must be 64, 128 or 256"; return false; }
  if (((c->flags & GMR_FLAG_HALF_WARP_FWD) && (c->flags & GMR_FLAG_WARP_STAGE_FWD)) ||
      ((c->flags & GMR_FLAG_HALF_WARP_BWD) && (c->flags & GMR_FLAG_WARP_STAGE_BWD))) {
    *why = "one compositing layout per direction";
    return false;
  }
  if ((c->flags & GMR_FLAG_DETERMINISTIC) && (c->flags & (GMR_FLAG_HALF_WARP_BWD | GMR_FLAG_WARP_STAGE_BWD))) {
    *why = "the deterministic backward runs in the block-staged layout";
    return false;
  }
  if ((c->flags & (GMR_FLAG_WARP_STAGE_FWD | GMR_FLAG_WARP_STAGE_BWD)) && (c->flags & GMR_FLAG_PERSISTENT)) {
    *why = "the warp-staged layout runs one CTA per tile (no persistent grid)";
    return false;
  }
  if (c->flags & (GMR_FLAG_HALF_WARP_FWD | GMR_FLAG_HALF_WARP_BWD)) {
    if (c->tile == 32 || (c->flags & GMR_FLAG_PERSISTENT)) {
      *why = "the half-warp layout needs 8x8 or 16x16 tiles and no persistent grid";
      return false;
    }
    if (c->tile == 16 && (((c->flags & GMR_FLAG_HALF_WARP_FWD) && c->threads == 64) ||
                          ((c->flags & GMR_FLAG_HALF_WARP_BWD) && c->threads_bwd == 64))) {
      *why = "the half-warp layout needs 128 or 256 threads per 16x16 tile";
      return false;
    }
  }
  if (c->cov_mode != GMR_COV_AREA && c->cov_mode != GMR_COV_EMBED_RAW) { *why = "bad cov_mode"; return false; }
  if (c->color_mode != GMR_COLOR_PER_FACE && c->color_mode != GMR_COLOR_PER_VERTEX && c->color_mode != GMR_COLOR_SH) {
    *why = "bad color_mode";
    return false;
  }
  if (c->color_mode == GMR_COLOR_SH && (c->sh_degree < 0 || c->sh_degree > 3)) {
    *why = "sh_degree must be 0..3";
    return false;
  }
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(c->bg[k])) { *why = "background must be finite"; return false; }
  return true;
}

// Grow a device buffer to at least `need` elements (geometric growth).
template <class T>
gmr_status grow(gmr_ctx* ctx, T** ptr, int64_t* cap, int64_t need, bool capturing, const char* what) {
  if (need <= *cap) return GMR_OK;
  if (capturing)
    return fail(ctx, GMR_ERR_STATE,
                std::string("workspace '") + what + "' must grow during stream capture; call gmr_reserve first");
  int64_t ncap = need + need / 4 + 1024;
  if (!within_limit(ctx, *ptr, (size_t)ncap * sizeof(T)))
    return fail(ctx, GMR_ERR_OOM, std::string("workspace '") + what + "' would exceed the workspace limit");
  T* p = nullptr;
  cudaError_t e = cudaMalloc((void**)&p, (size_t)ncap * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, GMR_ERR_OOM, std::string("cudaMalloc of workspace '") + what + "' failed");
  }
  track_alloc(ctx, p, (size_t)ncap * sizeof(T));
  if (*ptr) {
    track_free(ctx, *ptr);
    cudaFree(*ptr);
  }
  *ptr = p;
  *cap = ncap;
  return GMR_OK;
}

// (Re)allocates *ptr to exactly `count` elements (contents not kept).
template <class T>
gmr_status realloc_exact(gmr_ctx* ctx, T** ptr, int64_t count, const char* what) {
  T* p = nullptr;
  const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
  if (!within_limit(ctx, *ptr, bytes))
    return fail(ctx, GMR_ERR_OOM, std::string("workspace '") + what + "' would exceed the workspace limit");
  cudaError_t e = cudaMalloc((void**)&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, GMR_ERR_OOM, std::string("cudaMalloc of workspace '") + what + "' failed");
  }
  track_alloc(ctx, p, bytes);
  if (*ptr) {
    track_free(ctx, *ptr);
    cudaFree(*ptr);
  }
  *ptr = p;
  return GMR_OK;
}

// All per-record buffers are sized from one capacity (cap_records records).
gmr_status ensure_records(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_records) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "record workspace must grow during stream capture; call gmr_reserve");
  const int64_t cap = n + n / 4 + 1024;
  gmr_status s;
  if ((s = realloc_exact(ctx, &w.rec_uq, 2 * cap, "rec_uq")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.rec_rect, cap, "rec_rect")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.rec_ntiles, cap, "rec_ntiles")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.rec_key, cap, "rec_key")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.rec_grad, 2 * cap, "rec_grad")) != GMR_OK) return s;
  w.cap_records = cap;
  return GMR_OK;
}

// Per-record colours and colour gradient sums of the view-dependent colour.
gmr_status ensure_sh(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_sh_records) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "colour workspace must grow during stream capture; call gmr_reserve");
  const int64_t cap = n + n / 4 + 1024;
  gmr_status s;
  if ((s = realloc_exact(ctx, &w.rec_col, cap, "rec_col")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.rec_cgrad, cap, "rec_cgrad")) != GMR_OK) return s;
  w.cap_sh_records = cap;
  return GMR_OK;
}

gmr_status ensure_scratch(gmr_ctx* ctx, int64_t n_items, bool capturing) {
  Workspace& w = ctx->ws;
  return grow<uint32_t>(ctx, &w.scan_tmp, &w.cap_scan, gmr::scan_block_sums_needed(n_items), capturing, "scan_tmp");
}

// Per-tile counts, scanned starts and ranges. The counts must be zero at the
// start of every forward; a fresh allocation is cleared here.
// Zero-fills a freshly allocated buffer and waits for it, so that work on any
// stream (blocking or not) sees the zeros.
gmr_status zero_new(gmr_ctx* ctx, void* p, size_t bytes, const char* what) {
  cudaError_t e = cudaMemset(p, 0, bytes);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return GMR_OK;
}

// The loss partials (`slots` doubles): slot 0 is the loss kernels' ticket
// counter, zero between calls.
gmr_status ensure_loss(gmr_ctx* ctx, int64_t slots, bool capturing) {
  double* before = ctx->ws.loss_part;
  gmr_status st = grow<double>(ctx, &ctx->ws.loss_part, &ctx->ws.cap_loss, slots, capturing, "loss_part");
  if (st != GMR_OK || ctx->ws.loss_part == before) return st;
  return zero_new(ctx, ctx->ws.loss_part, sizeof(double), "loss_part");
}

gmr_status ensure_tiles(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n > w.cap_tiles) {
    if (capturing) return fail(ctx, GMR_ERR_STATE, "tile workspace must grow during stream capture; call gmr_reserve");
    const int64_t cap = n + n / 4 + 1024;
    gmr_status s;
    if ((s = realloc_exact(ctx, &w.tile_count, cap, "tile_count")) != GMR_OK) return s;
    if ((s = realloc_exact(ctx, &w.tile_start, cap, "tile_start")) != GMR_OK) return s;
    if ((s = realloc_exact(ctx, &w.tile_range, cap, "tile_range")) != GMR_OK) return s;
    if ((s = realloc_exact(ctx, &w.long_tiles, cap, "long_tiles")) != GMR_OK) return s;
    if ((s = realloc_exact(ctx, &w.tile_order, gmr::kTileClasses * cap, "tile_order")) != GMR_OK) return s;
    if ((s = realloc_exact(ctx, &w.tile_desc, cap, "tile_desc")) != GMR_OK) return s;
    if ((s = zero_new(ctx, w.tile_count, sizeof(uint32_t) * (size_t)cap, "tile_count")) != GMR_OK) return s;
    w.cap_tiles = cap;
  }
  return ensure_scratch(ctx, n, capturing);
}

gmr_status ensure_pairs(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_pairs) return GMR_OK;
  if (n >= (int64_t)(1 << 30) - 4096) return fail(ctx, GMR_ERR_CAPACITY, "more than 2^30 (tile, Gaussian) pairs");
  if (capturing) return fail(ctx, GMR_ERR_STATE, "pair workspace must grow during stream capture; call gmr_reserve");
  const int64_t cap = std::min<int64_t>(n + n / 4 + 4096, (int64_t)(1 << 30) - 4096);
  gmr_status s;
  for (int b = 0; b < 2; ++b)
    if ((s = realloc_exact(ctx, &w.pair_key[b], cap, "pair_key")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.pair_face, cap, "pair_face")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.pair_quad, cap, "pair_quad")) != GMR_OK) return s;
  w.cap_pairs = cap;
  return GMR_OK;
}

// Split binning: the 8x8 compositing descriptors (4 per binning tile) and
// ranges (one per 8x8 tile).
gmr_status ensure_split_tiles(gmr_ctx* ctx, int64_t n_btiles, int64_t n_tiles, bool capturing) {
  Workspace& w = ctx->ws;
  const int64_t need = std::max<int64_t>(4 * n_btiles, n_tiles);
  if (need <= w.cap_split_tiles) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "tile workspace must grow during stream capture; call gmr_reserve");
  const int64_t cap = need + need / 4 + 1024;
  gmr_status s;
  if ((s = realloc_exact(ctx, &w.tile_desc_c, cap, "tile_desc_c")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.tile_range_c, cap, "tile_range_c")) != GMR_OK) return s;
  w.cap_split_tiles = cap;
  return GMR_OK;
}

// Split binning: the quadrants' lists (4 face ids per pair slot).
gmr_status ensure_split_pairs(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_split_pairs) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "pair workspace must grow during stream capture; call gmr_reserve");
  gmr_status s = realloc_exact(ctx, &w.pair_face_c, n, "pair_face_c");
  if (s == GMR_OK) w.cap_split_pairs = n;
  return s;
}

// GMR_FLAG_DETERMINISTIC: the records' first pair slots.
gmr_status ensure_det_records(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_det_records) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "slot workspace must grow during stream capture; call gmr_reserve");
  const int64_t cap = n + n / 4 + 1024;
  gmr_status s = realloc_exact(ctx, &w.rec_slot, cap, "rec_slot");
  if (s == GMR_OK) w.cap_det_records = cap;
  return s;
}

// GMR_FLAG_DETERMINISTIC: the pair slots' sums (3 float4 per slot, as many
// slots as the pair buffers hold).
gmr_status ensure_det_pairs(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_det_pairs) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "pair-sum workspace must grow during stream capture; call gmr_reserve");
  gmr_status s = realloc_exact(ctx, &w.pair_grad, 3 * n, "pair_grad");
  if (s == GMR_OK) w.cap_det_pairs = n;
  return s;
}

// GMR_FLAG_DETERMINISTIC: the vertex-to-face incidence list and the faces'
// corner shares.
gmr_status ensure_det_mesh(gmr_ctx* ctx, int64_t V, int64_t F, bool capturing) {
  Workspace& w = ctx->ws;
  gmr_status s;
  if (V > w.cap_det_verts) {
    if (capturing) return fail(ctx, GMR_ERR_STATE, "vertex workspace must grow during stream capture; call gmr_reserve");
    const int64_t cap = V + V / 4 + 1024;
    if ((s = realloc_exact(ctx, &w.v_off, cap + 1, "v_off")) != GMR_OK) return s;
    if ((s = realloc_exact(ctx, &w.v_cur, cap, "v_cur")) != GMR_OK) return s;
    w.cap_det_verts = cap;
  }
  if (F > w.cap_det_faces) {
    if (capturing) return fail(ctx, GMR_ERR_STATE, "face workspace must grow during stream capture; call gmr_reserve");
    const int64_t cap = F + F / 4 + 1024;
    if ((s = realloc_exact(ctx, &w.v_inc, 3 * cap, "v_inc")) != GMR_OK) return s;
    if ((s = realloc_exact(ctx, &w.corner_grad, 4 * cap, "corner_grad")) != GMR_OK) return s;
    w.cap_det_faces = cap;
  }
  return GMR_OK;
}

// face_col and face_grad share one capacity.
gmr_status ensure_faces(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_faces) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "face workspace must grow during stream capture; call gmr_reserve");
  const int64_t cap = n + n / 4 + 1024;
  gmr_status s;
  if ((s = realloc_exact(ctx, &w.face_col, cap, "face_col")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.face_grad, cap, "face_grad")) != GMR_OK) return s;
  w.cap_faces = cap;
  return GMR_OK;
}

gmr_status ensure_pixels(gmr_ctx* ctx, int64_t n, bool capturing) {
  Workspace& w = ctx->ws;
  if (n <= w.cap_pixels) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "pixel workspace must grow during stream capture; call gmr_reserve");
  const int64_t cap = n + n / 4 + 1024;
  gmr_status s;
  if ((s = realloc_exact(ctx, &w.pix_T, cap, "pix_T")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.pix_last, cap, "pix_last")) != GMR_OK) return s;
  if ((s = realloc_exact(ctx, &w.pix_ncontrib, 2 * cap, "pix_ncontrib")) != GMR_OK) return s;
  w.cap_pixels = cap;
  return GMR_OK;
}

gmr_status ensure_views(gmr_ctx* ctx, int32_t C, bool capturing) {
  Workspace& w = ctx->ws;
  if (C <= w.cap_views) return GMR_OK;
  if (capturing) return fail(ctx, GMR_ERR_STATE, "view table must grow during stream capture");
  int64_t cap = w.cap_views;
  gmr_status s = grow<ViewInfo>(ctx, &w.views, &cap, C, false, "views");
  if (s != GMR_OK) return s;
  w.cap_views = (int32_t)cap;
  if (ctx->views_pinned) cudaFreeHost(ctx->views_pinned);
  ctx->views_pinned = nullptr;
  cudaError_t e = cudaMallocHost((void**)&ctx->views_pinned, (size_t)cap * sizeof(ViewInfo));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocHost(views)");
  ctx->views_pinned_cap = (int32_t)cap;
  return GMR_OK;
}

// NVTX range names of the stages (GMR_STAGE_* order), for profilers that
// filter or group kernels by range (ncu --nvtx --nvtx-include "gmr:raster_bwd/").
const char* const kStageRange[GMR_NUM_STAGES] = {"gmr:project", "gmr:scan", "gmr:bin", "gmr:raster_fwd",
                                                 "gmr:loss", "gmr:raster_bwd", "gmr:project_bwd"};

// Brackets one stage with an NVTX range (host side, around the stage's
// launches; a no-op unless a profiling tool is attached) and, when profiling
// is on, with events.
struct StageTimer {
  gmr_ctx* ctx;
  int stage;
  cudaStream_t s;
  bool on;
  unsigned flags;
  StageTimer(gmr_ctx* c, int st, cudaStream_t strm, const gmr_config& cfg)
      : ctx(c), stage(st), s(strm),
        on((cfg.flags & GMR_FLAG_PROFILE) && c->stage_ev[0] != nullptr &&
           (cfg.profile_stages == 0u || ((cfg.profile_stages >> st) & 1u))),
        flags(0) {
    nvtxRangePushA(kStageRange[st]);
    if (!on) return;
    // under stream capture the records must become event-record nodes of the
    // graph (external events), not capture-internal dependencies
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      flags = cudaEventRecordExternal;
    cudaEventRecordWithFlags(ctx->stage_ev[2 * stage], s, flags);
  }
  ~StageTimer() {
    if (on) {
      cudaEventRecordWithFlags(ctx->stage_ev[2 * stage + 1], s, flags);
      ctx->stage_mask |= 1u << stage;
    }
    nvtxRangePop();
  }
};


bool same_cams(const std::vector<gmr_camera>& a, const gmr_camera* b, int32_t C) {
  return (int32_t)a.size() == C && std::memcmp(a.data(), b, sizeof(gmr_camera) * (size_t)C) == 0;
}

gmr_status check_cams(gmr_ctx* ctx, const gmr_camera* cams, int32_t C) {
  for (int32_t c = 0; c < C; ++c) {
    const gmr_camera& k = cams[c];
    if (k.width <= 0 || k.height <= 0 || k.width > (1 << 20) || k.height > (1 << 20))
      return fail(ctx, GMR_ERR_INVALID_ARG, "camera " + std::to_string(c) + ": bad image size");
    // tile coordinates are packed in 16 bits in the projection's records
    const int64_t ts = ctx->cfg.tile;
    if ((k.width + ts - 1) / ts > 65536 || (k.height + ts - 1) / ts > 65536)
      return fail(ctx, GMR_ERR_INVALID_ARG, "camera " + std::to_string(c) + ": more than 65536 tiles per side");
    const float* f = &k.R[0];
    for (int q = 0; q < 16; ++q)
      if (!std::isfinite(f[q])) return fail(ctx, GMR_ERR_INVALID_ARG, "camera " + std::to_string(c) + ": non-finite");
    if (!std::isfinite(k.znear)) return fail(ctx, GMR_ERR_INVALID_ARG, "camera znear non-finite");
  }
  return GMR_OK;
}

// Split binning: 8x8 compositing tiles binned as 16x16 (then each sorted
// list split into its quadrants), except for the deterministic backward,
// whose pair slots follow the compositing tiles.
bool split_binning(const gmr_config& c) { return c.tile == 8 && !(c.flags & GMR_FLAG_DETERMINISTIC); }
// (the sort keys carry the quadrants below the face id: face << 4 | quadrants)
constexpr int64_t kSplitMaxFaces = int64_t(1) << 28;

// Builds the view table (tile and pixel bases) for the configured tile size
// and the binning grid.
void build_views(gmr_ctx* ctx, const gmr_camera* cams, int32_t C, int64_t* n_tiles, int64_t* n_pixels,
                 int64_t* n_btiles) {
  ctx->views.resize(C);
  int64_t tb = 0, pb = 0, bb = 0;
  int ts = ctx->cfg.tile;
  const int bs = split_binning(ctx->cfg) ? 2 * ts : ts;
  for (int32_t c = 0; c < C; ++c) {
    ViewInfo& v = ctx->views[c];
    std::memcpy(v.R, cams[c].R, sizeof(v.R));
    std::memcpy(v.t, cams[c].t, sizeof(v.t));
    v.fx = cams[c].fx; v.fy = cams[c].fy; v.cx = cams[c].cx; v.cy = cams[c].cy; v.znear = cams[c].znear;
    for (int q = 0; q < 3; ++q)  // camera centre -R^T t
      v.o[q] = (float)-((double)v.R[q] * v.t[0] + (double)v.R[3 + q] * v.t[1] + (double)v.R[6 + q] * v.t[2]);
    v.W = cams[c].width; v.H = cams[c].height;
    v.tiles_x = (v.W + ts - 1) / ts;
    v.tiles_y = (v.H + ts - 1) / ts;
    v.tile_base = (int32_t)tb;
    v.btiles_x = (v.W + bs - 1) / bs;
    v.btiles_y = (v.H + bs - 1) / bs;
    v.btile_base = (int32_t)bb;
    v.pix_base = pb;
    tb += (int64_t)v.tiles_x * v.tiles_y;
    bb += (int64_t)v.btiles_x * v.btiles_y;
    pb += (int64_t)v.W * v.H;
  }
  *n_tiles = tb;
  *n_pixels = pb;
  *n_btiles = bb;
}

}  // namespace

extern "C" {

const char* gmr_status_string(gmr_status s) {
  switch (s) {
    case GMR_OK: return "GMR_OK";
    case GMR_ERR_INVALID_ARG: return "GMR_ERR_INVALID_ARG";
    case GMR_ERR_CUDA: return "GMR_ERR_CUDA";
    case GMR_ERR_OOM: return "GMR_ERR_OOM";
    case GMR_ERR_CAPACITY: return "GMR_ERR_CAPACITY";
    case GMR_ERR_TIMEOUT: return "GMR_ERR_TIMEOUT";
    case GMR_ERR_STATE: return "GMR_ERR_STATE";
  }
  return "GMR_UNKNOWN";
}

gmr_status gmr_config_default(gmr_config* cfg) {
  if (!cfg) return GMR_ERR_INVALID_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->tile = 16;
  cfg->threads = 128;
  cfg->threads_bwd = 128;
  cfg->batch = 256;
  cfg->cov_mode = GMR_COV_AREA;
  cfg->color_mode = GMR_COLOR_PER_FACE;
  cfg->flags = GMR_FLAG_SYNC_CHECK;
  return GMR_OK;
}

gmr_status gmr_create(const gmr_config* cfg, gmr_ctx** out) {
  if (!out) return GMR_ERR_INVALID_ARG;
  *out = nullptr;
  gmr_config c;
  if (cfg) c = *cfg; else gmr_config_default(&c);
  std::string why;
  if (!valid_config(&c, &why)) return GMR_ERR_INVALID_ARG;
  gmr_ctx* ctx = new gmr_ctx();
  ctx->cfg = c;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->ws.counters, sizeof(Counters));
  if (e == cudaSuccess) e = cudaMemset(ctx->ws.counters, 0, sizeof(Counters));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->counters_pinned, sizeof(Counters));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->upload_done, cudaEventDisableTiming);
  for (int k = 0; k < 2 * GMR_NUM_STAGES && e == cudaSuccess; ++k) e = cudaEventCreate(&ctx->stage_ev[k]);
  if (e != cudaSuccess) {
    cudaGetLastError();
    gmr_destroy(ctx);
    return GMR_ERR_CUDA;
  }
  *out = ctx;
  return GMR_OK;
}

gmr_status gmr_destroy(gmr_ctx* ctx) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  Workspace& w = ctx->ws;
  void* bufs[] = {w.rec_uq, w.rec_rect, w.rec_ntiles, w.rec_key, w.rec_grad, w.rec_col, w.rec_cgrad,
                  w.face_col,
                  w.face_grad, w.pix_T, w.pix_last, w.pix_ncontrib, w.tile_count, w.tile_start, w.tile_range, w.long_tiles,
                  w.tile_order, w.tile_desc,
                  w.pair_key[0], w.pair_key[1], w.pair_face, w.scan_tmp, w.loss_part, w.views, w.counters, w.reg_scratch,
                  w.rec_slot, w.pair_grad, w.v_off, w.v_cur, w.v_inc, w.corner_grad, w.pair_face_c, w.tile_desc_c,
                  w.tile_range_c, w.pair_quad, w.verts4};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (ctx->views_pinned) cudaFreeHost(ctx->views_pinned);
  if (ctx->counters_pinned) cudaFreeHost(ctx->counters_pinned);
  if (ctx->upload_done) cudaEventDestroy(ctx->upload_done);
  for (int k = 0; k < 2 * GMR_NUM_STAGES; ++k)
    if (ctx->stage_ev[k]) cudaEventDestroy(ctx->stage_ev[k]);
  delete ctx;
  return GMR_OK;
}

gmr_status gmr_set_config(gmr_ctx* ctx, const gmr_config* cfg) {
  if (!ctx || !cfg) return fail(ctx, GMR_ERR_INVALID_ARG, "null argument");
  std::string why;
  if (!valid_config(cfg, &why)) return fail(ctx, GMR_ERR_INVALID_ARG, why);
  ctx->cfg = *cfg;
  ctx->fwd_valid = false;
  ctx->grads_zero = false;
  ctx->cams.clear();  // tile bases depend on the tile size
  return GMR_OK;
}

const char* gmr_last_error(const gmr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

gmr_status gmr_image_offsets(const gmr_camera* cams, int32_t C, int64_t* offsets) {
  if (!cams || !offsets || C < 0) return GMR_ERR_INVALID_ARG;
  int64_t p = 0;
  for (int32_t c = 0; c < C; ++c) {
    offsets[c] = p;
    p += (int64_t)cams[c].width * cams[c].height;
  }
  offsets[C] = p;
  return GMR_OK;
}

gmr_status gmr_set_workspace_limit(gmr_ctx* ctx, int64_t max_bytes) {
  if (!ctx || max_bytes < 0) return fail(ctx, GMR_ERR_INVALID_ARG, "bad workspace limit");
  ctx->dev_limit = max_bytes;
  return GMR_OK;
}

gmr_status gmr_reserve(gmr_ctx* ctx, int64_t max_faces, int32_t max_views, int64_t max_pixels, int64_t max_pairs) {
  if (!ctx || max_faces < 0 || max_views < 0 || max_pixels < 0 || max_pairs < 0)
    return fail(ctx, GMR_ERR_INVALID_ARG, "bad reserve sizes");
  // growing the buffers that hold the last forward's state drops that state
  struct Invalidate {
    gmr_ctx* c;
    int64_t before;
    ~Invalidate() {
      if (c->dev_bytes != before) {
        c->fwd_valid = false;
        c->grads_zero = false;
      }
    }
  } inval{ctx, ctx->dev_bytes};
  gmr_status s;
  if ((s = ensure_records(ctx, max_faces * (int64_t)max_views, false)) != GMR_OK) return s;
  if (ctx->cfg.color_mode == GMR_COLOR_SH && (s = ensure_sh(ctx, max_faces * (int64_t)max_views, false)) != GMR_OK)
    return s;
  if ((s = ensure_faces(ctx, max_faces, false)) != GMR_OK) return s;
  if ((s = grow<float4>(ctx, &ctx->ws.verts4, &ctx->ws.cap_verts4, 3 * max_faces, false, "verts4")) != GMR_OK)
    return s;
  if ((s = ensure_pixels(ctx, max_pixels, false)) != GMR_OK) return s;
  // tiles: at most one per tile-sized block plus one ragged tile per row and
  // column of each view (sides up to 16384 px; a larger view grows the
  // buffers in its forward)
  const int64_t ts = ctx->cfg.tile;
  int64_t mt = max_pixels / (ts * ts) + 2 * (int64_t)max_views * (16384 / ts) + 16;
  if ((s = ensure_tiles(ctx, mt, false)) != GMR_OK) return s;
  if ((s = ensure_views(ctx, max_views, false)) != GMR_OK) return s;
  if ((s = ensure_pairs(ctx, max_pairs, false)) != GMR_OK) return s;
  if (split_binning(ctx->cfg)) {
    // binning tiles of 16 px: fewer than the 8x8 tiles
    if ((s = ensure_split_tiles(ctx, mt, mt, false)) != GMR_OK) return s;
    if ((s = ensure_split_pairs(ctx, 4 * ctx->ws.cap_pairs, false)) != GMR_OK) return s;
  }
  if (ctx->cfg.flags & GMR_FLAG_DETERMINISTIC) {
    if ((s = ensure_det_records(ctx, max_faces * (int64_t)max_views, false)) != GMR_OK) return s;
    if ((s = ensure_det_pairs(ctx, ctx->ws.cap_pairs, false)) != GMR_OK) return s;
    if ((s = ensure_det_mesh(ctx, 3 * max_faces, max_faces, false)) != GMR_OK) return s;
  }
  return ensure_loss(ctx, std::max<int64_t>(gmr::l2_loss_partials_needed(3 * max_pixels), 1 + mt * 4), false);
}

gmr_status gmr_convert(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F,
                       const float* rgb, const float* opacity, float* means, float* cov, float* face_rgb,
                       float* face_opacity, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (V < 0 || F < 0) return fail(ctx, GMR_ERR_INVALID_ARG, "negative size");
  if (F > 0 && (!verts || !faces || V == 0)) return fail(ctx, GMR_ERR_INVALID_ARG, "null verts/faces");
  if (face_rgb && !rgb && F > 0) return fail(ctx, GMR_ERR_INVALID_ARG, "face_rgb requested without rgb");
  if (face_rgb && ctx->cfg.color_mode == GMR_COLOR_SH)
    return fail(ctx, GMR_ERR_INVALID_ARG, "face_rgb: with GMR_COLOR_SH the colour depends on the view");
  cudaStream_t s = (cudaStream_t)stream;
  GMR_CUDA(ctx, gmr::launch_convert(verts, V, faces, F, rgb, opacity, ctx->cfg.cov_mode, ctx->cfg.color_mode, means,
                                    cov, face_rgb, face_opacity, ctx->ws.counters, s, &ctx->launches));
  return GMR_OK;
}

namespace {

gmr_status render_fwd(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F, const float* rgb,
                      const float* opacity, const gmr_camera* cams, int32_t C, float* images, float* t_final,
                      gmr::FwdLoss fl, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  ctx->fwd_valid = false;
  ctx->grads_zero = false;
  if (V < 0 || F < 0) return fail(ctx, GMR_ERR_INVALID_ARG, "negative size");
  if (C < 1 || C > gmr::kMaxViews) return fail(ctx, GMR_ERR_INVALID_ARG, "C must be in [1, 65535]");
  if (!cams || !images) return fail(ctx, GMR_ERR_INVALID_ARG, "null cams or images");
  if (F > 0 && (!verts || !faces || !rgb || V == 0)) return fail(ctx, GMR_ERR_INVALID_ARG, "null mesh input");
  if ((int64_t)F * C >= (int64_t)0x7fffffff) return fail(ctx, GMR_ERR_INVALID_ARG, "views x faces >= 2^31");
  gmr_status st = check_cams(ctx, cams, C);
  if (st != GMR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  unsigned long long cap_id = 0;
  GMR_CUDA(ctx, cudaStreamGetCaptureInfo(s, &cap_status, &cap_id));
  const bool capturing = cap_status != cudaStreamCaptureStatusNone;
  const gmr_config& cfg = ctx->cfg;
  Workspace& w = ctx->ws;

  // view table
  const bool cams_same = same_cams(ctx->cams, cams, C);
  if (!cams_same && capturing)
    return fail(ctx, GMR_ERR_STATE, "cameras differ from the previous call during stream capture");
  int64_t n_tiles, n_pixels, n_btiles;
  build_views(ctx, cams, C, &n_tiles, &n_pixels, &n_btiles);
  const bool split = split_binning(cfg);
  if (split && F >= kSplitMaxFaces) return fail(ctx, GMR_ERR_INVALID_ARG, "8x8 tiles need fewer than 2^28 faces");
  if (n_tiles >= (int64_t)0x7fffffff) return fail(ctx, GMR_ERR_INVALID_ARG, "too many tiles");
  const int64_t n_rec = (int64_t)F * C;

  // workspace
  if ((st = ensure_views(ctx, C, capturing)) != GMR_OK) return st;
  if ((st = ensure_records(ctx, n_rec, capturing)) != GMR_OK) return st;
  if ((st = ensure_faces(ctx, F, capturing)) != GMR_OK) return st;
  if ((st = grow<float4>(ctx, &w.verts4, &w.cap_verts4, V, capturing, "verts4")) != GMR_OK) return st;
  if ((st = ensure_pixels(ctx, n_pixels, capturing)) != GMR_OK) return st;
  if ((st = ensure_tiles(ctx, n_tiles, capturing)) != GMR_OK) return st;
  if (cfg.color_mode == GMR_COLOR_SH && (st = ensure_sh(ctx, n_rec, capturing)) != GMR_OK) return st;
  if ((cfg.flags & GMR_FLAG_DETERMINISTIC) && (st = ensure_det_records(ctx, n_rec, capturing)) != GMR_OK) return st;
  if (split && (st = ensure_split_tiles(ctx, n_btiles, n_tiles, capturing)) != GMR_OK) return st;
  if (fl.target) {
    // one float per forward warp after slot 0 (gmr_l2_loss's ticket counter)
    const int64_t n_warp_sums = n_tiles * (ctx->cfg.threads / 32);
    if ((st = ensure_loss(ctx, 1 + (n_warp_sums + 1) / 2, capturing)) != GMR_OK) return st;
    fl.part = reinterpret_cast<float*>(w.loss_part + 1);
  }

  if (!cams_same) {
    GMR_CUDA(ctx, cudaEventSynchronize(ctx->upload_done));
    std::memcpy(ctx->views_pinned, ctx->views.data(), sizeof(ViewInfo) * (size_t)C);
    GMR_CUDA(ctx, cudaMemcpyAsync(w.views, ctx->views_pinned, sizeof(ViewInfo) * (size_t)C, cudaMemcpyHostToDevice, s));
    GMR_CUDA(ctx, cudaEventRecord(ctx->upload_done, s));
    ctx->cams.assign(cams, cams + C);
  }

  // S1-S3: conversion + projection per (view, face), per-face colour and
  // opacity, pair counts and in-tile ranks; tile segments = exclusive scan of
  // the per-tile counts (which it returns to zero), total pairs. With
  // SYNC_CHECK, a pair total beyond the pair buffers grows them and runs the
  // two stages again (the first run's pair scratch was incomplete).
  for (int attempt = 0;; ++attempt) {
    // counters: pair total and slots, forward and backward evaluation counts
    GMR_CUDA(ctx, cudaMemsetAsync(w.counters, 0, gmr::kStepCountersBytes, s));
    {
      StageTimer t(ctx, GMR_STAGE_PROJECT, s, cfg);
      GMR_CUDA(ctx, gmr::launch_project(verts, V, faces, F, rgb, opacity, cfg.color_mode, cfg.sh_degree, w.views, C,
                                        cfg.tile, split ? 1 : 0, cfg.cov_mode,
                                        (cfg.flags & GMR_FLAG_DETERMINISTIC) != 0, w, s, &ctx->launches));
    }
    {
      StageTimer t(ctx, GMR_STAGE_SCAN, s, cfg);
      GMR_CUDA(ctx, gmr::scan_exclusive(w.tile_count, n_btiles, w.tile_start, &w.counters->n_pairs,
                                        w.scan_tmp, w.tile_order, w.counters->n_class, s, &ctx->launches));
    }
    if (!(cfg.flags & GMR_FLAG_SYNC_CHECK) || capturing) break;
    GMR_CUDA(ctx, cudaMemcpyAsync(&ctx->counters_pinned->n_pairs, &w.counters->n_pairs, sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, s));
    GMR_CUDA(ctx, cudaStreamSynchronize(s));
    const int64_t P = ctx->counters_pinned->n_pairs;
    if (P <= w.cap_pairs) break;
    if (attempt > 0) return fail(ctx, GMR_ERR_STATE, "pair total changed between two identical projections");
    if ((st = ensure_pairs(ctx, P, false)) != GMR_OK) return st;
  }
  // S4-S6: keys to segment start + rank, per-tile sort by (depth, face),
  // ranges
  if (split && (st = ensure_split_pairs(ctx, 4 * w.cap_pairs, capturing)) != GMR_OK) return st;
  {
    StageTimer t(ctx, GMR_STAGE_BIN, s, cfg);
    GMR_CUDA(ctx, gmr::launch_bin_pairs(w, n_rec, F, w.views, C, n_btiles, split, s, &ctx->launches));
    if (split) GMR_CUDA(ctx, gmr::launch_split_quads(w, w.views, n_btiles, s, &ctx->launches));
  }
  // S7: compositing
  {
    StageTimer t(ctx, GMR_STAGE_RASTER_FWD, s, cfg);
    uint32_t* nc = (cfg.flags & GMR_FLAG_DEBUG_COUNTS) ? w.pix_ncontrib : nullptr;
    GMR_CUDA(ctx, gmr::launch_raster_fwd(cfg.tile, cfg.threads, cfg.batch, (cfg.flags & GMR_FLAG_PERSISTENT) != 0,
                                         (cfg.flags & GMR_FLAG_HALF_WARP_FWD) ? 1 : (cfg.flags & GMR_FLAG_WARP_STAGE_FWD) ? 2 : 0,
                                         cfg.color_mode == GMR_COLOR_SH, w, split ? w.tile_desc_c : w.tile_desc,
                                         split ? 4 * n_btiles : n_tiles, split ? w.pair_face_c : w.pair_face,
                                         w.views, C, F, n_tiles, cfg.bg, images, t_final, nc, fl, s,
                                         &ctx->launches));
  }

  ctx->fwd_valid = true;
  ctx->grads_zero = true;  // by the projection kernel
  ctx->grads_zero_capture = capturing ? cap_id : 0;
  ctx->verts = verts; ctx->faces = faces; ctx->rgb = rgb; ctx->opacity = opacity;
  ctx->V = V; ctx->F = F; ctx->C = C;
  ctx->n_tiles = n_tiles; ctx->n_pixels = n_pixels;
  ctx->n_btiles = n_btiles; ctx->split = split;
  ctx->fwd_cfg = cfg;
  return GMR_OK;
}

}  // namespace

gmr_status gmr_render_fwd(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F,
                          const float* rgb, const float* opacity, const gmr_camera* cams, int32_t C, float* images,
                          float* t_final, gmr_stream stream) {
  return render_fwd(ctx, verts, V, faces, F, rgb, opacity, cams, C, images, t_final, gmr::FwdLoss{}, stream);
}

gmr_status gmr_render_fwd_l2(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F,
                             const float* rgb, const float* opacity, const gmr_camera* cams, int32_t C,
                             float* images, float* t_final, const float* target, float* dL_dimg, double* loss,
                             gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (!target || !dL_dimg || !loss) return fail(ctx, GMR_ERR_INVALID_ARG, "null target, dL_dimg or loss");
  gmr::FwdLoss fl;
  fl.target = target;
  fl.grad = dL_dimg;
  fl.loss = loss;
  return render_fwd(ctx, verts, V, faces, F, rgb, opacity, cams, C, images, t_final, fl, stream);
}

gmr_status gmr_render_bwd(gmr_ctx* ctx, const float* dL_dimages, float* dL_dverts, float* dL_drgb,
                          float* dL_dopacity, int32_t accumulate, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (!dL_dimages) return fail(ctx, GMR_ERR_INVALID_ARG, "null dL_dimages");
  return gmr_render_bwd_ex(ctx, dL_dimages, nullptr, dL_dverts, dL_drgb, dL_dopacity, accumulate, stream);
}

gmr_status gmr_silhouette_bce(gmr_ctx* ctx, const float* t_final, const float* mask, int64_t n, float weight,
                              float* dL_dtfinal, double* loss, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!t_final || !mask || !dL_dtfinal)) || !loss)
    return fail(ctx, GMR_ERR_INVALID_ARG, "bad silhouette loss arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  GMR_CUDA(ctx, cudaStreamIsCapturing(s, &cap_status));
  gmr_status st = ensure_loss(ctx, gmr::bce_partials_needed(n), cap_status != cudaStreamCaptureStatusNone);
  if (st != GMR_OK) return st;
  GMR_CUDA(ctx, gmr::launch_silhouette_bce(t_final, mask, n, weight, dL_dtfinal, loss, ctx->ws.loss_part,
                                           ctx->ws.cap_loss, s, &ctx->launches));
  return GMR_OK;
}

namespace {

// The backward of the last forward from dL/dimages (or, with images and
// target, from the squared-error loss formed inside the compositing
// backward, whose sum goes to *loss) and dL/dT_final.
gmr_status render_bwd(gmr_ctx* ctx, const float* dL_dimages, const float* dL_dtfinal, const float* images,
                      const float* target, double* loss, float* dL_dverts, float* dL_drgb, float* dL_dopacity,
                      int32_t accumulate, gmr_stream stream) {
  if (!ctx->fwd_valid) return fail(ctx, GMR_ERR_STATE, "gmr_render_bwd without a preceding gmr_render_fwd");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = ctx->ws;
  const gmr_config& cfg = ctx->fwd_cfg;
  const int32_t F = ctx->F, C = ctx->C, V = ctx->V;
  gmr::BwdLoss bl;
  const int64_t n_cta_sums = ctx->n_tiles;
  if (images) {
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    GMR_CUDA(ctx, cudaStreamIsCapturing(s, &cap_status));
    gmr_status st = ensure_loss(ctx, 1 + (n_cta_sums + 1) / 2, cap_status != cudaStreamCaptureStatusNone);
    if (st != GMR_OK) return st;
    bl.img = images;
    bl.target = target;
    bl.part = reinterpret_cast<float*>(w.loss_part + 1);
  }
  const int64_t n_rec = (int64_t)F * C;
  const bool det = (cfg.flags & GMR_FLAG_DETERMINISTIC) != 0;
  if (det) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GMR_CUDA(ctx, cudaStreamIsCapturing(s, &cs));
    const bool capt = cs != cudaStreamCaptureStatusNone;
    gmr_status st;
    if ((st = ensure_det_pairs(ctx, w.cap_pairs, capt)) != GMR_OK) return st;
    if ((st = ensure_det_mesh(ctx, V, F, capt)) != GMR_OK) return st;
  }
  // The record and face gradient sums, the evaluation counter and the
  // persistent grid's cursor start at
  // zero: the forward's projection zeroed them if this backward follows it
  // directly (in stream order, or in the same graph capture); else here.
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  unsigned long long cap_id = 0;
  GMR_CUDA(ctx, cudaStreamGetCaptureInfo(s, &cap_status, &cap_id));
  const unsigned long long cap_now = cap_status != cudaStreamCaptureStatusNone ? cap_id : 0;
  const bool zeroed = ctx->grads_zero && ctx->grads_zero_capture == cap_now;
  ctx->grads_zero = false;
  if (!zeroed) {
    if (n_rec > 0) GMR_CUDA(ctx, cudaMemsetAsync(w.rec_grad, 0, sizeof(float4) * 2 * (size_t)n_rec, s));
    if (cfg.color_mode == GMR_COLOR_SH) {
      if (n_rec > 0) GMR_CUDA(ctx, cudaMemsetAsync(w.rec_cgrad, 0, sizeof(float4) * (size_t)n_rec, s));
    } else if (F > 0) {
      GMR_CUDA(ctx, cudaMemsetAsync(w.face_grad, 0, sizeof(float4) * (size_t)F, s));
    }
    GMR_CUDA(ctx, cudaMemsetAsync(&w.counters->evals_bwd, 0, gmr::kBwdCountersBytes, s));
  }
  // outputs the projection backward accumulates into: zeroed by the
  // compositing backward's CTAs (or here, when it has no tiles)
  gmr::BwdZero bz;
  if (!accumulate && !det) {  // (the deterministic gather writes every vertex)
    int k = 0;
    if (dL_dverts && V > 0) { bz.p[k] = dL_dverts; bz.n[k++] = 3 * (int64_t)V; }
    if (dL_drgb && cfg.color_mode == GMR_COLOR_PER_VERTEX && V > 0) { bz.p[k] = dL_drgb; bz.n[k++] = 3 * (int64_t)V; }
    if (ctx->n_tiles <= 0) {
      for (int z = 0; z < k; ++z) GMR_CUDA(ctx, cudaMemsetAsync(bz.p[z], 0, sizeof(float) * (size_t)bz.n[z], s));
      bz = gmr::BwdZero{};
    }
  }
  // S8: compositing backward
  {
    StageTimer t(ctx, GMR_STAGE_RASTER_BWD, s, cfg);
    GMR_CUDA(ctx, gmr::launch_raster_bwd(cfg.tile, cfg.threads_bwd, cfg.batch, (cfg.flags & GMR_FLAG_PERSISTENT) != 0,
                                         (cfg.flags & GMR_FLAG_HALF_WARP_BWD) ? 1 : (cfg.flags & GMR_FLAG_WARP_STAGE_BWD) ? 2 : 0,
                                         cfg.color_mode == GMR_COLOR_SH, det, w,
                                         ctx->split ? w.tile_desc_c : w.tile_desc,
                                         ctx->split ? 4 * ctx->n_btiles : ctx->n_tiles,
                                         ctx->split ? w.pair_face_c : w.pair_face, w.views, C, F, ctx->n_tiles, cfg.bg,
                                         dL_dimages, dL_dtfinal, bl, bz, s, &ctx->launches));
  }
  if (images) {  // the loss: sum of the warps' partial sums
    StageTimer t(ctx, GMR_STAGE_LOSS, s, cfg);
    if (n_cta_sums > 0) {
      GMR_CUDA(ctx, gmr::launch_sum_floats(bl.part, n_cta_sums, 1.0, loss, s, &ctx->launches));
    } else {
      GMR_CUDA(ctx, cudaMemsetAsync(loss, 0, sizeof(double), s));
    }
  }
  // S9: projection + conversion backward, vertex scatter
  {
    StageTimer t(ctx, GMR_STAGE_PROJECT_BWD, s, cfg);
    GMR_CUDA(ctx, gmr::launch_project_bwd(ctx->verts, V, ctx->faces, F, w.views, C, cfg.cov_mode, cfg.color_mode,
                                          cfg.sh_degree, ctx->rgb, ctx->opacity, det, w, dL_dverts, dL_drgb,
                                          dL_dopacity, accumulate, s, &ctx->launches));
  }
  return GMR_OK;
}

}  // namespace

gmr_status gmr_render_bwd_ex(gmr_ctx* ctx, const float* dL_dimages, const float* dL_dtfinal, float* dL_dverts,
                             float* dL_drgb, float* dL_dopacity, int32_t accumulate, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (!dL_dimages && !dL_dtfinal) return fail(ctx, GMR_ERR_INVALID_ARG, "null dL_dimages and dL_dtfinal");
  return render_bwd(ctx, dL_dimages, dL_dtfinal, nullptr, nullptr, nullptr, dL_dverts, dL_drgb, dL_dopacity,
                    accumulate, stream);
}

gmr_status gmr_render_bwd_l2(gmr_ctx* ctx, const float* images, const float* target, double* loss,
                             const float* dL_dtfinal, float* dL_dverts, float* dL_drgb, float* dL_dopacity,
                             int32_t accumulate, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (!images || !target || !loss) return fail(ctx, GMR_ERR_INVALID_ARG, "null images, target or loss");
  return render_bwd(ctx, nullptr, dL_dtfinal, images, target, loss, dL_dverts, dL_drgb, dL_dopacity, accumulate,
                    stream);
}

gmr_status gmr_l2_loss(gmr_ctx* ctx, const float* img, const float* target, int64_t n, float* dL_dimg,
                       double* loss, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!img || !target || !dL_dimg)) || !loss)
    return fail(ctx, GMR_ERR_INVALID_ARG, "bad loss arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  GMR_CUDA(ctx, cudaStreamIsCapturing(s, &cap_status));
  gmr_status st = ensure_loss(ctx, gmr::l2_loss_partials_needed(n), cap_status != cudaStreamCaptureStatusNone);
  if (st != GMR_OK) return st;
  StageTimer t(ctx, GMR_STAGE_LOSS, s, ctx->cfg);
  GMR_CUDA(ctx, gmr::launch_l2_loss(img, target, n, dL_dimg, loss, ctx->ws.loss_part, ctx->ws.cap_loss, s,
                                    &ctx->launches));
  return GMR_OK;
}

gmr_status gmr_adam_step(gmr_ctx* ctx, float* params, const float* grads, float* m, float* v, int64_t n,
                         int32_t group, float lr, float beta1, float beta2, float eps, int32_t step,
                         gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (n < 0 || (group != 1 && group != 3) || n % group != 0 || step < 1 ||
      (n > 0 && (!params || !grads || !m || !v)))
    return fail(ctx, GMR_ERR_INVALID_ARG, "bad Adam arguments");
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return fail(ctx, GMR_ERR_INVALID_ARG, "bad Adam hyper-parameters");
  GMR_CUDA(ctx, gmr::launch_adam(params, grads, m, v, n, group, lr, beta1, beta2, eps, step, (cudaStream_t)stream,
                                 &ctx->launches));
  return GMR_OK;
}

gmr_status gmr_mesh_regularizers(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F,
                                 float w_edge, float w_lap, float* dL_dverts, double* losses, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (V < 1 || F < 1 || !verts || !faces || !losses) return fail(ctx, GMR_ERR_INVALID_ARG, "bad regulariser arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  GMR_CUDA(ctx, cudaStreamIsCapturing(s, &cap_status));
  // 2 leading floats hold the mean edge length (a double)
  gmr_status st = grow<float>(ctx, &ctx->ws.reg_scratch, &ctx->ws.cap_reg, 2 + gmr::regularizer_scratch_floats(V, F),
                              cap_status != cudaStreamCaptureStatusNone, "reg_scratch");
  if (st != GMR_OK) return st;
  GMR_CUDA(ctx, gmr::launch_regularizers(verts, V, faces, F, w_edge, w_lap, dL_dverts, losses,
                                         ctx->ws.reg_scratch + 2, reinterpret_cast<double*>(ctx->ws.reg_scratch), s,
                                         &ctx->launches));
  return GMR_OK;
}

gmr_status gmr_chamfer(gmr_ctx* ctx, const float* a, int64_t na, const float* b, int64_t nb, double* out,
                       gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (na < 1 || nb < 1 || !a || !b || !out) return fail(ctx, GMR_ERR_INVALID_ARG, "bad chamfer arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  GMR_CUDA(ctx, cudaStreamIsCapturing(s, &cap_status));
  // per-point minima as floats after slot 0 (gmr_l2_loss's ticket counter)
  gmr_status st = ensure_loss(ctx, 1 + (na + nb + 1) / 2, cap_status != cudaStreamCaptureStatusNone);
  if (st != GMR_OK) return st;
  GMR_CUDA(ctx, gmr::launch_chamfer(a, na, b, nb, reinterpret_cast<float*>(ctx->ws.loss_part + 1), out, s,
                                    &ctx->launches));
  return GMR_OK;
}

gmr_status gmr_get_device_status(gmr_ctx* ctx, gmr_stream stream, uint32_t* status) {
  if (!ctx || !status) return GMR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GMR_CUDA(ctx, cudaMemcpyAsync(&ctx->counters_pinned->status, &ctx->ws.counters->status, sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, s));
  GMR_CUDA(ctx, cudaMemsetAsync(&ctx->ws.counters->status, 0, sizeof(uint32_t), s));
  GMR_CUDA(ctx, cudaStreamSynchronize(s));
  *status = ctx->counters_pinned->status;
  return GMR_OK;
}

gmr_status gmr_get_stats(gmr_ctx* ctx, gmr_stream stream, gmr_stats* out) {
  if (!ctx || !out) return GMR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GMR_CUDA(ctx, cudaMemcpyAsync(ctx->counters_pinned, ctx->ws.counters, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  GMR_CUDA(ctx, cudaStreamSynchronize(s));
  out->n_records = (int64_t)ctx->F * ctx->C;
  out->n_pairs = ctx->counters_pinned->n_pairs;
  out->n_tiles = ctx->n_tiles;
  out->n_pixels = ctx->n_pixels;
  out->evals_fwd = (int64_t)ctx->counters_pinned->evals_fwd;
  out->evals_bwd = (int64_t)ctx->counters_pinned->evals_bwd;
  out->contribs = (int64_t)ctx->counters_pinned->contribs;
  out->launches = ctx->launches;
  out->pair_capacity = ctx->ws.cap_pairs;
  out->workspace_bytes = ctx->dev_bytes;
  return GMR_OK;
}

gmr_status gmr_get_stage_times(gmr_ctx* ctx, gmr_stream stream, float* ms) {
  if (!ctx || !ms) return GMR_ERR_INVALID_ARG;
  GMR_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  for (int k = 0; k < GMR_NUM_STAGES; ++k) {
    ms[k] = -1.0f;
    if (!(ctx->stage_mask & (1u << k))) continue;
    float t = -1.0f;
    if (cudaEventElapsedTime(&t, ctx->stage_ev[2 * k], ctx->stage_ev[2 * k + 1]) == cudaSuccess) ms[k] = t;
    else cudaGetLastError();
  }
  return GMR_OK;
}

gmr_status gmr_debug_forward_state(gmr_ctx* ctx, uint32_t* depth_bits, int32_t* rects, uint32_t* tile_ids,
                                   uint32_t* face_ids, int64_t cap, uint32_t* ranges, float* rec_u, float* rec_conic,
                                   uint32_t* n_last, uint32_t* n_contrib, int64_t* n_pairs, gmr_stream stream) {
  if (!ctx) return GMR_ERR_INVALID_ARG;
  if (!ctx->fwd_valid) return fail(ctx, GMR_ERR_STATE, "no forward state");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = ctx->ws;
  const int64_t n_rec = (int64_t)ctx->F * ctx->C;
  GMR_CUDA(ctx, cudaMemcpyAsync(&ctx->counters_pinned->n_pairs, &w.counters->n_pairs, sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, s));
  GMR_CUDA(ctx, cudaStreamSynchronize(s));
  int64_t P = ctx->counters_pinned->n_pairs;
  if (n_pairs) *n_pairs = P;
  if (n_rec > 0 && (rects || rec_conic))
    GMR_CUDA(ctx, gmr::launch_debug_records(w, n_rec, rects, rec_conic, s, &ctx->launches));
  if (depth_bits && n_rec > 0)
    GMR_CUDA(ctx, cudaMemcpyAsync(depth_bits, w.rec_key, sizeof(uint32_t) * (size_t)n_rec, cudaMemcpyDeviceToDevice,
                                  s));
  if (rec_u && n_rec > 0)
    GMR_CUDA(ctx, cudaMemcpy2DAsync(rec_u, sizeof(float4), w.rec_uq, 2 * sizeof(float4), sizeof(float4), (size_t)n_rec,
                                    cudaMemcpyDeviceToDevice, s));
  if (P > w.cap_pairs) return fail(ctx, GMR_ERR_CAPACITY, "pair buffer overflowed in the forward");
  if (ctx->split) {
    // the 8x8 tiles' lists sit at 4 start + q n of their binning tile's
    // segment: gathered here, in tile order, into the packed form
    const int64_t nt = ctx->n_tiles;
    std::vector<uint2> rg((size_t)std::max<int64_t>(nt, 1));
    std::vector<uint32_t> pf((size_t)std::max<int64_t>(4 * P, 1));
    if (nt > 0)
      GMR_CUDA(ctx, cudaMemcpyAsync(rg.data(), w.tile_range_c, sizeof(uint2) * (size_t)nt, cudaMemcpyDeviceToHost, s));
    if (P > 0)
      GMR_CUDA(ctx, cudaMemcpyAsync(pf.data(), w.pair_face_c, sizeof(uint32_t) * 4 * (size_t)P, cudaMemcpyDeviceToHost,
                                    s));
    GMR_CUDA(ctx, cudaStreamSynchronize(s));
    std::vector<uint2> crg((size_t)std::max<int64_t>(nt, 1));
    std::vector<uint32_t> tid, fid;
    for (int64_t g = 0; g < nt; ++g) {
      const uint32_t b = (uint32_t)fid.size();
      for (uint32_t i = rg[g].x; i < rg[g].y; ++i) {
        tid.push_back((uint32_t)g);
        fid.push_back(pf[i]);
      }
      crg[g] = fid.size() > b ? make_uint2(b, (uint32_t)fid.size()) : make_uint2(0u, 0u);
    }
    const int64_t P8 = (int64_t)fid.size();
    if (n_pairs) *n_pairs = P8;
    if ((tile_ids || face_ids) && P8 > cap) return fail(ctx, GMR_ERR_CAPACITY, "cap smaller than the pair count");
    if (tile_ids && P8 > 0)
      GMR_CUDA(ctx, cudaMemcpyAsync(tile_ids, tid.data(), sizeof(uint32_t) * (size_t)P8, cudaMemcpyHostToDevice, s));
    if (face_ids && P8 > 0)
      GMR_CUDA(ctx, cudaMemcpyAsync(face_ids, fid.data(), sizeof(uint32_t) * (size_t)P8, cudaMemcpyHostToDevice, s));
    if (ranges && nt > 0)
      GMR_CUDA(ctx, cudaMemcpyAsync(ranges, crg.data(), sizeof(uint2) * (size_t)nt, cudaMemcpyHostToDevice, s));
    GMR_CUDA(ctx, cudaStreamSynchronize(s));  // (the host vectors go out of scope)
    tile_ids = face_ids = ranges = nullptr;
  }
  if ((tile_ids || face_ids) && P > cap) return fail(ctx, GMR_ERR_CAPACITY, "cap smaller than the pair count");
  if (tile_ids && P > 0) GMR_CUDA(ctx, gmr::launch_expand_tiles(w.tile_range, ctx->n_tiles, tile_ids, s, &ctx->launches));
  if (face_ids && P > 0)
    GMR_CUDA(ctx, cudaMemcpyAsync(face_ids, w.pair_face, sizeof(uint32_t) * (size_t)P, cudaMemcpyDeviceToDevice, s));
  if (ranges)
    GMR_CUDA(ctx, cudaMemcpyAsync(ranges, w.tile_range, sizeof(uint2) * (size_t)ctx->n_tiles,
                                  cudaMemcpyDeviceToDevice, s));
  if (n_last && ctx->n_pixels > 0)
    GMR_CUDA(ctx, cudaMemcpyAsync(n_last, w.pix_last, sizeof(uint32_t) * (size_t)ctx->n_pixels,
                                  cudaMemcpyDeviceToDevice, s));
  if (n_contrib && ctx->n_pixels > 0) {
    if (!(ctx->fwd_cfg.flags & GMR_FLAG_DEBUG_COUNTS))
      return fail(ctx, GMR_ERR_STATE, "contributor counts need GMR_FLAG_DEBUG_COUNTS in the forward");
    GMR_CUDA(ctx, cudaMemcpyAsync(n_contrib, w.pix_ncontrib, sizeof(uint32_t) * (size_t)ctx->n_pixels,
                                  cudaMemcpyDeviceToDevice, s));
    GMR_CUDA(ctx, cudaMemcpyAsync(n_contrib + ctx->n_pixels, w.pix_ncontrib + w.cap_pixels,
                                  sizeof(uint32_t) * (size_t)ctx->n_pixels, cudaMemcpyDeviceToDevice, s));
  }
  return GMR_OK;
}

}  // extern "C"
