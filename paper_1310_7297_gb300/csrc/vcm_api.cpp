// vcm_api.cpp -- host runtime behind the C ABI of include/vcm.h.
//
// Canonicalises requests onto the 2^-10 m lattice (exact integer rounding of
// patch centres and viewpoints), owns the device scene and its grid index,
// lays out launch descriptors, runs single requests on the caller's stream,
// batches uneven requests into one persistent launch (replayed from a CUDA
// graph), and schedules asynchronous requests onto execution slots with
// memory-budget admission (continuous batching).
#include "vcm_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace vcm;

struct Ticket;   // one asynchronous request (defined below)

namespace {

thread_local std::string t_err;

// An NVTX range over a host stage (visible to nsys / ncu --nvtx; a no-op
// when no tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

vcm_status fail(vcm_status s, const char *fmt, ...)
{
    char buf[768];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? VCM_E_NOMEM : VCM_E_CUDA,             \
                        "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,       \
                        __LINE__);                                                              \
    } while (0)

constexpr int64_t kLimitUnits = int64_t(1) << 24;
constexpr double kUnitsPerM = 1024.0;
constexpr double kPi = 3.14159265358979323846;

bool to_units(float x, int64_t &u)
{
    if (!std::isfinite(x))
        return false;
    const double d = (double)x * kUnitsPerM;   // exact for a float
    if (d != std::floor(d) || std::fabs(d) > (double)kLimitUnits)
        return false;
    u = (int64_t)d;
    return true;
}

// nearest integer to num / den (den > 0), halves away from zero
int64_t round_half_away(int64_t num, int64_t den)
{
    if (num >= 0)
        return (2 * num + den) / (2 * den);
    return -((2 * (-num) + den) / (2 * den));
}

float units_to_float(int64_t u) { return (float)((double)u / kUnitsPerM); }

int pow2_at_least(int x)
{
    int p = 1;
    while (p < x)
        p <<= 1;
    return p;
}

// ---------------------------------------------------------------------------
// canonical request
// ---------------------------------------------------------------------------

struct Canon {
    int dims = 3;
    int au = 0, an = 1, aw = 2, perm = 0;
    float sn = 1.f, p_n = 0.f;
    int nu = 1, nw = 1, P = 1, words = 1;
    float measure = 0.f;
    int nx = 1, ny = 1, nl = 1;
    std::vector<float> u_coord, w_coord, x_coord, y_coord, z_coord;
    float u_min = 0, u_max = 0, w_min = 0, w_max = 0;
    int levels = 16;
    float v_ref = 0.f;
    unsigned flags = 0;
    int cone = 0;
    float cone_c = 0.f, cone_a[3] = {0.f, 0.f, 0.f};
    long long n_vp = 0;
    size_t out_bytes() const
    {
        size_t b = (size_t)n_vp * (sizeof(float) + 1);
        if (flags & VCM_EMIT_BITS)
            b += (size_t)n_vp * words * sizeof(uint32_t);
        return b;
    }
    int coord_count() const { return nu + nw + nx + ny + nl; }
};

int perm_index(int a0, int a1, int a2)
{
    static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int i = 0; i < 6; ++i)
        if (P[i][0] == a0 && P[i][1] == a1 && P[i][2] == a2)
            return i;
    return -1;
}

vcm_status canonicalise_grid(const vcm_request *r, Canon &c);

// Viewer-centric request: the viewer is a one-point "target" in the world
// frame (u = x, n = y, w = z), the object size S is kept in `measure`.
vcm_status canonicalise_viewer(const vcm_request *r, Canon &c)
{
    c.au = 0;
    c.an = 1;
    c.aw = 2;
    c.perm = 0;
    c.sn = 1.f;
    c.nu = c.nw = c.P = c.words = 1;
    int64_t cu[3] = {0, 0, 0};
    for (int k = 0; k < c.dims; ++k)
        if (!to_units(r->center[k], cu[k]))
            return fail(VCM_E_ARG, "viewer center[%d] is not a finite lattice value within 16384 m", k);
    int64_t S = 0;
    if (!to_units(r->width, S) || S <= 0)
        return fail(VCM_E_ARG, "width (object size S) must be a positive lattice value");
    c.u_coord.assign(1, units_to_float(cu[0]));
    c.w_coord.assign(1, units_to_float(cu[2]));
    c.p_n = units_to_float(cu[1]);
    c.u_min = c.u_max = c.u_coord[0];
    c.w_min = c.w_max = c.w_coord[0];
    c.measure = units_to_float(S);
    return canonicalise_grid(r, c);
}

vcm_status canonicalise(const vcm_request *r, Canon &c)
{
    Range range("vcm canonicalise");
    if (!r)
        return fail(VCM_E_ARG, "request is NULL");
    if (r->dims != 2 && r->dims != 3)
        return fail(VCM_E_ARG, "dims must be 2 or 3 (got %d)", r->dims);
    c.dims = r->dims;
    if (r->flags & ~(uint32_t)(VCM_EMIT_BITS | VCM_STRICT | VCM_VIEWER | VCM_TWO_SIDED | VCM_CACHE_BITS))
        return fail(VCM_E_ARG, "unknown flag bits 0x%x", r->flags);
    if ((r->flags & VCM_CACHE_BITS) && (r->flags & VCM_VIEWER))
        return fail(VCM_E_ARG, "VCM_CACHE_BITS and VCM_VIEWER exclude each other");
    if ((r->flags & VCM_STRICT) && (r->flags & VCM_VIEWER))
        return fail(VCM_E_ARG, "VCM_STRICT and VCM_VIEWER exclude each other");
    if ((r->flags & VCM_TWO_SIDED) && (r->flags & VCM_VIEWER))
        return fail(VCM_E_ARG, "VCM_TWO_SIDED and VCM_VIEWER exclude each other");
    if (!std::isfinite(r->fov_deg) || r->fov_deg < 0.f)
        return fail(VCM_E_ARG, "fov_deg must be finite and >= 0");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(r->gaze[k]))
            return fail(VCM_E_ARG, "gaze must be finite");
    const bool cone = r->fov_deg > 0.f && r->fov_deg < 360.f;
    c.flags = r->flags;
    if (r->flags & VCM_VIEWER) {
        if (cone)
            return fail(VCM_E_ARG, "a field of view applies to target-centric requests only");
        return canonicalise_viewer(r, c);
    }
    if (r->axis_u < 0 || r->axis_u > 5 || r->normal < 0 || r->normal > 5)
        return fail(VCM_E_ARG, "axis codes must be 0..5");
    c.au = r->axis_u >> 1;
    c.an = r->normal >> 1;
    c.sn = (r->normal & 1) ? -1.f : 1.f;
    const int64_t su = (r->axis_u & 1) ? -1 : 1;
    int64_t sw = 1;
    if (c.dims == 3) {
        if (r->axis_w < 0 || r->axis_w > 5)
            return fail(VCM_E_ARG, "axis_w must be 0..5");
        c.aw = r->axis_w >> 1;
        sw = (r->axis_w & 1) ? -1 : 1;
        if (c.au == c.an || c.au == c.aw || c.an == c.aw)
            return fail(VCM_E_ARG, "axis_u, axis_w and normal must be three different axes");
    } else {
        c.aw = 2;
        if (c.au > 1 || c.an > 1 || c.au == c.an)
            return fail(VCM_E_ARG, "2D target: axis_u and normal must be x and y in some order");
    }
    c.perm = perm_index(c.au, c.an, c.aw);
    if (cone) {
        // the cone's cosine and unit axis, rounded once from double
        c.cone = 1;
        c.cone_c = (float)std::cos((double)r->fov_deg * kPi / 360.0);
        double g[3] = {r->gaze[0], r->gaze[1], c.dims == 3 ? r->gaze[2] : 0.0f};
        if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0)
            g[c.an] = (double)c.sn;
        const double len = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        for (int k = 0; k < 3; ++k)
            c.cone_a[k] = (float)(g[k] / len);
    }
    if (r->patches_u < 1 || r->patches_u > VCM_MAX_PATCHES_SIDE)
        return fail(VCM_E_ARG, "patches_u must be 1..%u", VCM_MAX_PATCHES_SIDE);
    c.nu = (int)r->patches_u;
    c.nw = 1;
    if (c.dims == 3) {
        if (r->patches_w < 1 || r->patches_w > VCM_MAX_PATCHES_SIDE)
            return fail(VCM_E_ARG, "patches_w must be 1..%u", VCM_MAX_PATCHES_SIDE);
        c.nw = (int)r->patches_w;
    }
    c.P = c.nu * c.nw;
    if ((unsigned)c.P > VCM_MAX_PATCHES)
        return fail(VCM_E_ARG, "at most %u patches", VCM_MAX_PATCHES);
    c.words = (c.P + 31) / 32;
    int64_t cu[3];
    for (int k = 0; k < 3; ++k) {
        if (c.dims == 2 && k == 2) {
            cu[k] = 0;
            continue;
        }
        if (!to_units(r->center[k], cu[k]))
            return fail(VCM_E_ARG, "center[%d] = %g is not a finite lattice value within 16384 m", k,
                        (double)r->center[k]);
    }
    int64_t W = 0, H = 0;
    if (!to_units(r->width, W) || W <= 0)
        return fail(VCM_E_ARG, "width must be a positive lattice value");
    if (c.dims == 3 && (!to_units(r->height, H) || H <= 0))
        return fail(VCM_E_ARG, "height must be a positive lattice value");
    // patch centres along u and w
    c.u_coord.resize(c.nu);
    for (int iu = 0; iu < c.nu; ++iu) {
        const int64_t Nu = c.nu;
        const int64_t v = round_half_away(2 * Nu * cu[c.au] + su * (2 * iu + 1 - Nu) * W, 2 * Nu);
        if (v < -kLimitUnits || v > kLimitUnits)
            return fail(VCM_E_ARG, "patch centre outside the coordinate limit");
        c.u_coord[iu] = units_to_float(v);
    }
    c.w_coord.assign(c.nw, 0.f);
    if (c.dims == 3) {
        for (int iw = 0; iw < c.nw; ++iw) {
            const int64_t Nw = c.nw;
            const int64_t v = round_half_away(2 * Nw * cu[c.aw] + sw * (2 * iw + 1 - Nw) * H, 2 * Nw);
            if (v < -kLimitUnits || v > kLimitUnits)
                return fail(VCM_E_ARG, "patch centre outside the coordinate limit");
            c.w_coord[iw] = units_to_float(v);
        }
    }
    c.p_n = units_to_float(cu[c.an]);
    c.u_min = *std::min_element(c.u_coord.begin(), c.u_coord.end());
    c.u_max = *std::max_element(c.u_coord.begin(), c.u_coord.end());
    c.w_min = *std::min_element(c.w_coord.begin(), c.w_coord.end());
    c.w_max = *std::max_element(c.w_coord.begin(), c.w_coord.end());
    {
        const double lu = (double)W / kUnitsPerM / c.nu;
        c.measure = (float)(c.dims == 3 ? lu * ((double)H / kUnitsPerM / c.nw) : lu);
    }
    return canonicalise_grid(r, c);
}

// The viewpoint grid, layers, colour levels and v_ref of a request.
vcm_status canonicalise_grid(const vcm_request *r, Canon &c)
{
    if (r->grid_nx < 1 || r->grid_ny < 1 || r->grid_nx > VCM_MAX_GRID_SIDE || r->grid_ny > VCM_MAX_GRID_SIDE)
        return fail(VCM_E_ARG, "grid_nx and grid_ny must be 1..%u", VCM_MAX_GRID_SIDE);
    c.nx = (int)r->grid_nx;
    c.ny = (int)r->grid_ny;
    int64_t o[2], s[2];
    for (int k = 0; k < 2; ++k) {
        if (!to_units(r->grid_origin[k], o[k]))
            return fail(VCM_E_ARG, "grid_origin[%d] is not a finite lattice value", k);
        if (!to_units(r->grid_step[k], s[k]) || s[k] <= 0)
            return fail(VCM_E_ARG, "grid_step[%d] must be a positive lattice value", k);
    }
    c.x_coord.resize(c.nx);
    c.y_coord.resize(c.ny);
    for (int i = 0; i < c.nx; ++i) {
        const int64_t v = round_half_away(2 * o[0] + (int64_t)(2 * i + 1) * s[0], 2);
        if (v < -kLimitUnits || v > kLimitUnits)
            return fail(VCM_E_ARG, "viewpoint x outside the coordinate limit");
        c.x_coord[i] = units_to_float(v);
    }
    for (int i = 0; i < c.ny; ++i) {
        const int64_t v = round_half_away(2 * o[1] + (int64_t)(2 * i + 1) * s[1], 2);
        if (v < -kLimitUnits || v > kLimitUnits)
            return fail(VCM_E_ARG, "viewpoint y outside the coordinate limit");
        c.y_coord[i] = units_to_float(v);
    }
    if (c.dims == 3) {
        if (r->n_layers < 1 || r->n_layers > VCM_MAX_LAYERS || !r->layer_z)
            return fail(VCM_E_ARG, "n_layers must be 1..%u with layer_z given", VCM_MAX_LAYERS);
        c.nl = (int)r->n_layers;
        c.z_coord.resize(c.nl);
        for (int l = 0; l < c.nl; ++l) {
            int64_t z;
            if (!to_units(r->layer_z[l], z))
                return fail(VCM_E_ARG, "layer_z[%d] is not a finite lattice value", l);
            c.z_coord[l] = units_to_float(z);
        }
    } else {
        c.nl = 1;
        c.z_coord.assign(1, 0.f);
    }
    if (r->color_levels < 2 || r->color_levels > 256)
        return fail(VCM_E_ARG, "color_levels must be 2..256");
    c.levels = (int)r->color_levels;
    if (!std::isfinite(r->v_ref))
        return fail(VCM_E_ARG, "v_ref must be finite");
    c.v_ref = r->v_ref;
    c.n_vp = (long long)c.nx * c.ny * c.nl;
    return VCM_OK;
}

// lane mapping and tiling of a canonical request under a launch shape
void fill_shape(const Canon &c, const vcm_tune &t, DevRequest &d)
{
    d.nuc = std::min(c.nu, 32);
    d.groups = 32 / d.nuc;
    d.col_passes = (c.nu + d.nuc - 1) / d.nuc;
    const int rows_per_lane = (c.nw + d.groups - 1) / d.groups;
    int k = pow2_at_least(std::min(rows_per_lane, 8));
    if (t.patch_k > 0)
        k = std::min(k, pow2_at_least(std::min<int>(t.patch_k, 8)));
    if (c.cone || (c.flags & VCM_TWO_SIDED))
        k = 8;   // the tile kernel sweeps these requests with its 8-row variant
    d.k_rows = k;
    d.row_passes = (c.nw + d.groups * k - 1) / (d.groups * k);
    // Work sharing: chunks of 32 open viewpoints, published from a tile
    // with at least 8 open.  Smaller chunks for requests with many patches
    // (about the same work per chunk) were slower: each chunk stages its
    // owner's candidate list again (100,000-box scene, 64 x 32 patches:
    // 8 viewpoints +7 %, 4 viewpoints +26 %; publishing from 4 open +0.5 %).
    d.chunk_vp = kChunkVp;
    d.min_publish = kMinPublish;
    d.tile_x = (int)std::max(1u, t.tile_x);
    d.tile_y = (int)std::max(1u, t.tile_y);
    d.tiles_x = (c.nx + d.tile_x - 1) / d.tile_x;
    d.tiles_y = (c.ny + d.tile_y - 1) / d.tile_y;
    d.n_tiles = d.tiles_x * d.tiles_y * c.nl;
}

// Scheduler thresholds, in viewpoint-patch segments: batches up to
// kSmallWork run on high-priority slots; a batch stops growing past
// kBatchWork (a request larger than that runs alone).
constexpr double kSmallWork = 2.0e8;
constexpr double kBatchWork = 1.0e9;

int tune_class(int P)
{
    if (P <= 32)
        return 0;
    if (P <= 128)
        return 1;
    if (P <= 512)
        return 2;
    if (P <= 2048)
        return 3;
    return 4;
}
constexpr int kTuneClasses = 5;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// pinned host pool
// ---------------------------------------------------------------------------

class PinnedPool {
  public:
    ~PinnedPool()
    {
        for (auto &kv : free_)
            cudaFreeHost(kv.second);
    }
    void *get(size_t bytes)
    {
        std::lock_guard<std::mutex> g(mu_);
        size_t want = std::max<size_t>(4096, (size_t)1 << (64 - __builtin_clzll((std::max<size_t>(bytes, 1) - 1) | 1)));
        auto it = free_.lower_bound(want);
        if (it != free_.end() && it->first <= 2 * want) {
            void *p = it->second;
            size_[p] = it->first;
            free_.erase(it);
            return p;
        }
        void *p = nullptr;
        if (cudaMallocHost(&p, want) != cudaSuccess)
            return nullptr;
        size_[p] = want;
        return p;
    }
    void put(void *p)
    {
        if (!p)
            return;
        std::lock_guard<std::mutex> g(mu_);
        auto it = size_.find(p);
        if (it == size_.end())
            return;
        free_.emplace(it->second, p);
        size_.erase(it);
    }

  private:
    std::mutex mu_;
    std::multimap<size_t, void *> free_;
    std::map<void *, size_t> size_;
};

// ---------------------------------------------------------------------------
// launch resources
// ---------------------------------------------------------------------------

// Descriptor arena of one launch: DevRequest[n] | tile prefix | viewpoint
// prefix | coordinates.  Built in pinned host memory, copied in one H2D.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t desc_copied = nullptr;
    char *d_desc = nullptr, *h_desc = nullptr;
    size_t desc_cap = 0;
    int *d_work = nullptr;
    int *d_spill = nullptr;
    size_t spill_cap = 0;   // ints
    int *d_spill_busy = nullptr;   // spill-region claims of one-tile launches
    size_t spill_busy_cap = 0;
    bool high_priority = false;
    vcm_stats *d_stats = nullptr;
    size_t stats_cap = 0;   // entries
    bool busy = false;
    // completion: the slot's waiter thread blocks on `done` (without any
    // lock held), then marks the in-flight group finished
    cudaEvent_t done = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;   // device time of the in-flight launch
    cudaEvent_t kernels_done = nullptr;       // its last kernel (before the result copies)
    cudaEvent_t t_chain = nullptr;            // where its wait for the launch before it ended
    bool chained = false;                     // t_chain recorded for the in-flight launch
    std::vector<std::shared_ptr<::Ticket>> inflight;
    bool posted = false;
    std::thread waiter;
    bool scheduler = false;   // one of the scheduler's slots (its scratch counts against the budget)
    size_t scratch = 0;       // bytes of scratch the slot holds
    // graphs of the device work of one batched launch, one per launch form
    // (0: one block per tile, 1: persistent with the chunk pass)
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    // everything a form's graph was captured with (parameters, buffers,
    // scene); an equal key replays the graph as it is
    std::vector<unsigned long long> key[2];
    // the parameters of the slot's previous launch of each form: a launch
    // equal to it is captured (it is likely to come again), others run
    // directly
    std::vector<unsigned long long> last_key[2];
};

struct Layout {
    size_t off_reqs, off_tiles, off_vps, off_coords, bytes;
    int total_tiles;
    long long total_vp;
    long long blocker_ints;   // tile positions of the requests in the blocker table
};

// Occlusion bits kept for recolouring (VCM_CACHE_BITS): a request's bits
// do not depend on its field of view, gaze, sides, strictness or colours,
// so a later request whose canonical target, patches and viewpoint grid are
// the same (scene unchanged) is served from them (Section IV-C).
struct CacheEntry {
    std::vector<float> key;        // canonical geometry (cache_key)
    unsigned long long scene_gen = 0;
    uint32_t *d_bits = nullptr;
    size_t bytes = 0;
    bool ready = false;            // the launch that fills it has completed
    int users = 0;                 // in-flight launches writing or reading it
    uint64_t last_use = 0;
};

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct vcm_ctx {
    int device = 0;
    int sm_count = 1;
    size_t budget = 0, used = 0;
    std::mutex mu;             // guards everything below except the scene during launches
    std::condition_variable cv;
    // scene
    int dims = 0;
    uint32_t n_boxes = 0;
    std::vector<float> h_lo, h_hi;   // n x 3
    float *d_lo = nullptr, *d_hi = nullptr;
    size_t lo_cap = 0, idx_box_cap = 0, idx_cell_cap = 0;   // allocated capacities (boxes, cells + 1)
    bool built = false;
    unsigned long long scene_gen = 0;   // bumped by every vcm_build
    float4 *d_perm[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int *d_cell_start = nullptr, *d_cell_of = nullptr, *d_count = nullptr, *d_cursor = nullptr, *d_order = nullptr;
    float4 *d_cell_lo = nullptr, *d_cell_hi = nullptr;
    unsigned *d_overhang = nullptr;
    DevScene scene{};
    // tuning
    vcm_tune tune[kTuneClasses];
    bool forced = false;
    vcm_tune forced_tune{};
    // launch slots
    Slot direct;                      // vcm_compute / vcm_compute_batch
    std::vector<std::unique_ptr<Slot>> slots;   // scheduler
    uint32_t max_batch = 64;
    cudaEvent_t ev_before = nullptr, ev_after = nullptr;   // optional timing of the tile kernel
    int *d_recolor_list = nullptr;   // vcm_recolor: viewpoints that need a measure, and their count
    int *d_recolor_n = nullptr;
    size_t recolor_cap = 0;
    PinnedPool pinned;
    cudaStream_t aux = nullptr;
    // scheduler
    std::deque<std::vector<std::shared_ptr<Ticket>>> queue;
    std::map<uint64_t, std::shared_ptr<Ticket>> tickets;
    uint64_t next_ticket = 1;
    std::thread worker;
    bool stop = false;
    int running_groups = 0;
    size_t scratch = 0;   // scratch held by the scheduler's slots (counted against the budget)
    Slot *last_launched = nullptr;   // the slot of the most recent scheduler launch
    // host-side fault injection (vcm_inject): launches with every spill
    // region held, and failing request-buffer allocations, still to come
    uint32_t inject_spill = 0, inject_alloc = 0;
    // occlusion bits kept for recolouring, least recently used first out
    std::vector<std::shared_ptr<CacheEntry>> cache;
    size_t cache_bytes = 0;
    uint64_t cache_clock = 0;
    // per-request metric lines (vcm_set_request_log) and the latencies of the
    // last kLatencyRing completed requests (vcm_latency_summary)
    std::mutex log_mu;
    FILE *req_log = nullptr;        // guarded by log_mu
    std::atomic<bool> log_on{false};
    std::vector<double> lat_ring;   // guarded by mu
    uint64_t lat_done = 0;
};

namespace {

enum TicketState { T_QUEUED, T_RUNNING, T_DONE, T_ERROR, T_CANCELLED };

}  // namespace

struct Ticket {
    uint64_t id = 0;
    Canon canon;
    vcm_tune shape{};
    TicketState state = T_QUEUED;
    vcm_status err = VCM_OK;
    std::string msg;
    float *d_v = nullptr;
    uint8_t *d_color = nullptr;
    uint32_t *d_bits = nullptr;
    float *h_v = nullptr;
    uint8_t *h_color = nullptr;
    uint32_t *h_bits = nullptr;
    vcm_stats *h_stats = nullptr;
    size_t bytes = 0;
    Slot *slot = nullptr;
    std::chrono::steady_clock::time_point t_submit, t_launch, t_done;
    double device_ms = 0.0;
    double launch_ms = 0.0;   // host time to enqueue its launch
    double chain_ms = 0.0;    // device wait for the launch before it
    uint32_t group_size = 0, form = 0;
    std::shared_ptr<CacheEntry> cache_fill;   // cached bits this request's launch writes
    std::shared_ptr<CacheEntry> cache_hit;    // cached bits it is recoloured from
};

namespace {

// 16 x 16 viewpoints per tile: with the chunk phase taking the open
// viewpoints of expensive tiles, larger tiles spread the cull (16 x 8 was
// 2 % slower on the 3D workload and the 100,000-box scene, 4 % on the
// 256-request mix; 32 x 8 and 32 x 16 were 40-90 % slower, 8 x 8 18 %).
// 448 staged boxes: at 6 and 7 blocks per SM, less shared memory leaves more
// L1 for the tile kernel's spilled registers (against 512: 100,000-box
// step -0.5 %, 5,000-box step -2.1 %, 256-request batch -0.4 %; 1,024 was
// 28 % slower on the 100,000-box scene).
vcm_tune default_tune()
{
    vcm_tune t;
    t.tile_x = 16;
    t.tile_y = 16;
    t.patch_k = 8;
    t.box_cap = 448;
    return t;
}

vcm_tune shape_for(vcm_ctx *ctx, const Canon &c)
{
    if (ctx->forced)
        return ctx->forced_tune;
    if (c.flags & VCM_VIEWER) {
        // one segment per cell: larger tiles spread the per-tile cull over
        // more cells (3D workload, 512 x 512 x 5 cells: 16 x 8 0.20 ms,
        // 32 x 8 0.14, 32 x 16 0.13, 32 x 32 0.16; 2,048 staged boxes slower)
        vcm_tune t{};
        t.tile_x = 32;
        t.tile_y = 16;
        t.patch_k = 8;
        t.box_cap = 512;
        return t;
    }
    return ctx->tune[tune_class(c.P)];
}

Layout layout_for(const std::vector<const Canon *> &cs, const std::vector<vcm_tune> &shapes)
{
    Layout L{};
    const size_t n = cs.size();
    L.off_reqs = 0;
    L.off_tiles = align_up(sizeof(DevRequest) * n, 256);
    L.off_vps = align_up(L.off_tiles + sizeof(int) * (n + 1), 256);
    L.off_coords = align_up(L.off_vps + sizeof(long long) * (n + 1), 256);
    size_t coords = 0;
    L.total_tiles = 0;
    L.total_vp = 0;
    L.blocker_ints = 0;
    for (size_t i = 0; i < n; ++i) {
        coords += cs[i]->coord_count();
        DevRequest d{};
        fill_shape(*cs[i], shapes[i], d);
        L.total_tiles += d.n_tiles;
        L.total_vp += cs[i]->n_vp;
        const long long pos = (long long)d.tiles_x * d.tiles_y;
        if (L.blocker_ints + pos <= kBlockerCap)   // fill_desc gives the same offsets
            L.blocker_ints += pos;
    }
    L.bytes = align_up(L.off_coords + sizeof(float) * coords, 256);
    return L;
}

// Fill the pinned descriptor arena (host side) for a launch.
void fill_desc(char *h, const char *d_base, const Layout &L, const std::vector<const Canon *> &cs,
               const std::vector<vcm_tune> &shapes, float *const *v, uint8_t *const *color,
               uint32_t *const *bits, vcm_stats *stats, int box_cap, bool blockers = true)
{
    const size_t n = cs.size();
    DevRequest *reqs = reinterpret_cast<DevRequest *>(h + L.off_reqs);
    int *tiles = reinterpret_cast<int *>(h + L.off_tiles);
    long long *vps = reinterpret_cast<long long *>(h + L.off_vps);
    float *coords = reinterpret_cast<float *>(h + L.off_coords);
    const float *d_coords = reinterpret_cast<const float *>(d_base + L.off_coords);
    size_t at = 0;
    int tp = 0;
    long long vp = 0, blk = 0;
    for (size_t i = 0; i < n; ++i) {
        const Canon &c = *cs[i];
        DevRequest d{};
        d.dims = c.dims;
        d.au = c.au; d.an = c.an; d.aw = c.aw; d.perm = c.perm;
        d.sn = c.sn; d.p_n = c.p_n;
        d.nu = c.nu; d.nw = c.nw; d.P = c.P; d.words = c.words;
        d.measure = c.measure;
        d.nx = c.nx; d.ny = c.ny; d.nl = c.nl;
        fill_shape(c, shapes[i], d);
        auto put = [&](const std::vector<float> &src) {
            const float *dp = d_coords + at;
            std::memcpy(coords + at, src.data(), sizeof(float) * src.size());
            at += src.size();
            return dp;
        };
        d.u_coord = put(c.u_coord);
        d.w_coord = put(c.w_coord);
        d.x_coord = put(c.x_coord);
        d.y_coord = put(c.y_coord);
        d.z_coord = put(c.z_coord);
        d.u_min = c.u_min; d.u_max = c.u_max; d.w_min = c.w_min; d.w_max = c.w_max;
        d.v_out = v[i];
        d.color_out = color ? color[i] : nullptr;
        d.bits_out = bits ? bits[i] : nullptr;
        d.stats = stats + i;
        d.v_ref_given = c.v_ref;
        d.levels = c.levels;
        d.flags = c.flags;
        d.box_cap = box_cap;
        d.cone = c.cone;
        d.cone_c = c.cone_c;
        for (int k = 0; k < 3; ++k)
            d.cone_a[k] = c.cone_a[k];
        // the request's tile positions in the blocker table (as layout_for counts them)
        d.blk_base = -1;
        const long long pos = (long long)d.tiles_x * d.tiles_y;
        if (blk + pos <= kBlockerCap) {
            if (blockers)
                d.blk_base = (int)blk;
            blk += pos;
        }
        reqs[i] = d;
        tiles[i] = tp;
        vps[i] = vp;
        tp += d.n_tiles;
        vp += c.n_vp;
    }
    tiles[n] = tp;
    vps[n] = vp;
}

// Device bytes of a slot's scratch.
size_t slot_bytes(const Slot &s)
{
    return s.desc_cap + (s.d_work ? kWorkBytes : 0) + (s.spill_cap + s.spill_busy_cap) * sizeof(int) +
           s.stats_cap * sizeof(vcm_stats);
}

// Scratch one scheduler slot needs for the current scene: the work arena,
// a spill list of n_boxes ints for every block that can be resident (at the
// smallest shared-memory size, the most blocks), their claim words, 256
// stats entries and 1 MB of descriptors.
size_t slot_scratch_need(const vcm_ctx *ctx)
{
    const size_t blocks = (size_t)tiles_blocks_per_sm(32) * (size_t)ctx->sm_count;
    return kWorkBytes + blocks * (std::max<uint32_t>(ctx->n_boxes, 1) + 1) * sizeof(int) + 256 * sizeof(vcm_stats) +
           ((size_t)1 << 20);
}

vcm_status ensure_slot_impl(vcm_ctx *ctx, Slot &s, size_t desc_bytes, size_t n_stats, int grid_blocks,
                            cudaStream_t sync_stream)
{
    if (s.scheduler) {
        // A scheduler slot takes its whole scratch for the scene at its
        // first launch (what admission charged: slot_scratch_need), so a
        // later, larger launch does not regrow it: a cudaFree would wait
        // for the device while the context lock is held.
        grid_blocks = std::max(grid_blocks, tiles_blocks_per_sm(32) * ctx->sm_count);
        desc_bytes = std::max<size_t>(desc_bytes, (size_t)1 << 19);
        n_stats = std::max<size_t>(n_stats, 256);
    }
    const size_t spill_need = (size_t)grid_blocks * std::max<uint32_t>(ctx->n_boxes, 1);
    const bool grow = desc_bytes > s.desc_cap || spill_need > s.spill_cap || n_stats > s.stats_cap ||
                      !s.d_work || (size_t)grid_blocks > s.spill_busy_cap;
    if (!grow)
        return VCM_OK;
    // the slot's buffers may still be read by queued work
    CUDA_TRY(cudaStreamSynchronize(sync_stream));
    if (s.stream && s.stream != sync_stream)
        CUDA_TRY(cudaStreamSynchronize(s.stream));
    if (!s.desc_copied)
        CUDA_TRY(cudaEventCreateWithFlags(&s.desc_copied, cudaEventDisableTiming));
    if (!s.d_work)   // tile-queue counters (zeroed by k_prologue) and the work-sharing arena
        CUDA_TRY(cudaMalloc(&s.d_work, kWorkBytes));
    if (desc_bytes > s.desc_cap) {
        size_t cap = std::max<size_t>(desc_bytes * 2, 1 << 16);
        if (s.d_desc) cudaFree(s.d_desc);
        if (s.h_desc) cudaFreeHost(s.h_desc);
        s.d_desc = nullptr;
        s.h_desc = nullptr;
        CUDA_TRY(cudaMalloc(&s.d_desc, cap));
        CUDA_TRY(cudaMallocHost(&s.h_desc, cap));
        s.desc_cap = cap;
        for (int f = 0; f < 2; ++f) {
            if (s.exec[f]) {
                cudaGraphExecDestroy(s.exec[f]);
                s.exec[f] = nullptr;
            }
            if (s.graph[f]) {
                cudaGraphDestroy(s.graph[f]);
                s.graph[f] = nullptr;
            }
        }
    }
    if (spill_need > s.spill_cap) {
        if (s.d_spill) cudaFree(s.d_spill);
        s.d_spill = nullptr;
        CUDA_TRY(cudaMalloc(&s.d_spill, spill_need * sizeof(int)));
        s.spill_cap = spill_need;
    }
    if ((size_t)grid_blocks > s.spill_busy_cap) {
        if (s.d_spill_busy) cudaFree(s.d_spill_busy);
        s.d_spill_busy = nullptr;
        CUDA_TRY(cudaMalloc(&s.d_spill_busy, (size_t)grid_blocks * sizeof(int)));
        // on the launch stream: the slots' streams do not wait for the legacy default stream
        CUDA_TRY(cudaMemsetAsync(s.d_spill_busy, 0, (size_t)grid_blocks * sizeof(int), sync_stream));
        s.spill_busy_cap = (size_t)grid_blocks;
    }
    if (n_stats > s.stats_cap) {
        size_t cap = std::max<size_t>(n_stats, 256);
        if (s.d_stats) cudaFree(s.d_stats);
        s.d_stats = nullptr;
        CUDA_TRY(cudaMalloc(&s.d_stats, cap * sizeof(vcm_stats)));
        s.stats_cap = cap;
    }
    return VCM_OK;
}

// Grow a slot's scratch as a launch needs it; a scheduler slot's bytes are
// kept in the context's count, which admission charges against the budget.
vcm_status ensure_slot(vcm_ctx *ctx, Slot &s, size_t desc_bytes, size_t n_stats, int grid_blocks,
                       cudaStream_t sync_stream)
{
    const vcm_status st = ensure_slot_impl(ctx, s, desc_bytes, n_stats, grid_blocks, sync_stream);
    const size_t now = slot_bytes(s);
    if (s.scheduler)
        ctx->scratch = ctx->scratch - s.scratch + now;
    s.scratch = now;
    return st;
}

// Staged boxes of a launch: the largest of its requests' shapes (at least
// 32, the smallest vcm_set_tune takes).
int launch_box_cap(const std::vector<vcm_tune> &shapes)
{
    uint32_t cap = 32;
    for (auto &t : shapes)
        cap = std::max(cap, t.box_cap);
    return (int)std::min<uint32_t>(cap, 5000);
}

// A launch with few tiles leaves SMs idle while its expensive tiles run
// (a tile is one block's work item): shrink the tiles, 16 x 16 -> 16 x 8 ->
// 8 x 8 -> 8 x 4, until the launch holds four waves of resident blocks.
// Measured on the 64 requests of the serving pool, each launched alone: the
// sum of their times 45.3 ms -> 26.1 ms (the best shape per request would
// give 25.7 ms); a 124 x 124 x 5 grid with 64 x 32 patches 3.28 -> 0.30 ms.
// Launches with many tiles (the 3D workloads, batches) keep their shapes.
void shrink_small_launch(vcm_ctx *ctx, const std::vector<const Canon *> &cs, std::vector<vcm_tune> &shapes)
{
    if (ctx->forced || cs.empty())
        return;
    const long long target = 4LL * tiles_blocks_per_sm(launch_box_cap(shapes)) * ctx->sm_count;
    for (;;) {
        long long total = 0;
        for (size_t i = 0; i < cs.size(); ++i) {
            DevRequest d{};
            fill_shape(*cs[i], shapes[i], d);
            total += d.n_tiles;
        }
        if (total >= target)
            return;
        bool any = false;
        for (auto &t : shapes) {
            if (t.tile_y >= t.tile_x && t.tile_y > 4) {
                t.tile_y /= 2;
                any = true;
            } else if (t.tile_x > 8) {
                t.tile_x /= 2;
                any = true;
            }
        }
        if (!any)
            return;
    }
}

int grid_blocks_for(vcm_ctx *ctx, int box_cap, int total_tiles)
{
    const int per_sm = tiles_blocks_per_sm(box_cap);
    return std::max(1, std::min(total_tiles, per_sm * ctx->sm_count));
}

struct Prepared {
    Layout L;
    int box_cap = 0;
    int blocks = 0;
    size_t n = 0;
    bool extra = false;   // a request is two-sided or has a field-of-view cone
    bool any_bits = false;   // a request emits occlusion bits
    bool tile_check = false;   // every request has many patches: whole-tile check
};

bool needs_extra(const Canon &c) { return c.cone || (c.flags & VCM_TWO_SIDED); }

// Host half of a launch: layout, scratch, and the descriptor arena filled in
// pinned memory.  `stats` must hold cs.size() entries.
vcm_status prepare_launch(vcm_ctx *ctx, Slot &s, const std::vector<const Canon *> &cs,
                          const std::vector<vcm_tune> &shapes_in, float *const *v, uint8_t *const *color,
                          uint32_t *const *bits, vcm_stats *stats, cudaStream_t sync_stream, Prepared &P,
                          bool adapt = true)
{
    Range range("vcm prepare launch");
    if (!ctx->built)
        return fail(VCM_E_STATE, "vcm_build has not been called for the current scene");
    std::vector<vcm_tune> shapes = shapes_in;
    if (adapt)
        shrink_small_launch(ctx, cs, shapes);
    P.L = layout_for(cs, shapes);
    P.box_cap = launch_box_cap(shapes);
    P.blocks = grid_blocks_for(ctx, P.box_cap, P.L.total_tiles);
    P.n = cs.size();
    P.extra = P.any_bits = false;
    P.tile_check = !cs.empty();
    for (const Canon *c : cs) {
        P.extra = P.extra || needs_extra(*c);
        P.any_bits = P.any_bits || (c->flags & VCM_EMIT_BITS);
        P.tile_check = P.tile_check && c->P >= kTileCheckMinPatches;
    }
    vcm_status st = ensure_slot(ctx, s, P.L.bytes, cs.size(), P.blocks, sync_stream);
    if (st != VCM_OK)
        return st;
    // the previous upload from h_desc must have completed before rewriting it
    CUDA_TRY(cudaEventSynchronize(s.desc_copied));
    fill_desc(s.h_desc, s.d_desc, P.L, cs, shapes, v, color, bits, stats, P.box_cap);
    return VCM_OK;
}

// Device half: descriptor upload, counters, bit buffers, the persistent tile
// kernel and the quantiser, in stream order.  The node sequence is the same
// for every launch, so a captured graph can be updated in place.
vcm_status record_launch(vcm_ctx *ctx, Slot &s, const Prepared &P, vcm_stats *stats, cudaStream_t stream,
                         bool timed = false, bool capturing = false, bool one_tile = false,
                         int claim_rounds = kClaimRounds, bool hold_spill = false,
                         cudaEvent_t after = nullptr)
{
    Range range("vcm record launch");
    CUDA_TRY(cudaMemcpyAsync(s.d_desc, s.h_desc, P.L.bytes, cudaMemcpyHostToDevice, stream));
    // An event recorded inside a stream capture cannot be waited on later;
    // a captured launch records it after the graph launch instead.
    if (!capturing)
        CUDA_TRY(cudaEventRecord(s.desc_copied, stream));

    const DevRequest *d_reqs = reinterpret_cast<const DevRequest *>(s.d_desc + P.L.off_reqs);
    const int *d_tiles = reinterpret_cast<const int *>(s.d_desc + P.L.off_tiles);
    const long long *d_vps = reinterpret_cast<const long long *>(s.d_desc + P.L.off_vps);
    (void)stats;   // the descriptors point into it; the prologue clears it
    CUDA_TRY(launch_prologue(d_reqs, (int)P.n, s.d_work, P.any_bits, stream));
    if (P.tile_check && P.L.blocker_ints > 0)   // no blocker recorded yet (-1)
        CUDA_TRY(cudaMemsetAsync(s.d_work + kWorkHeader + kBlockerOff, 0xFF, (size_t)P.L.blocker_ints * sizeof(int),
                                 stream));
    // the tile kernel starts after another launch's kernels (see launch_group)
    if (after) {
        CUDA_TRY(cudaStreamWaitEvent(stream, after, 0));
        if (!capturing && s.t_chain) {
            CUDA_TRY(cudaEventRecord(s.t_chain, stream));
            s.chained = true;
        }
    }
    // fault injection: every spill region already held (any nonzero word)
    if (hold_spill)
        CUDA_TRY(cudaMemsetAsync(s.d_spill_busy, 1, s.spill_busy_cap * sizeof(int), stream));
    if (timed && ctx->ev_before)
        CUDA_TRY(cudaEventRecord(ctx->ev_before, stream));
    CUDA_TRY(launch_tiles(ctx->scene, d_reqs, d_tiles, (int)P.n, P.L.total_tiles, s.d_work, s.d_spill,
                          P.blocks, P.box_cap, P.extra, P.tile_check, stream, one_tile, s.d_spill_busy,
                          /*share=*/true, claim_rounds));
    if (timed && ctx->ev_after)
        CUDA_TRY(cudaEventRecord(ctx->ev_after, stream));
    if (hold_spill)
        CUDA_TRY(cudaMemsetAsync(s.d_spill_busy, 0, s.spill_busy_cap * sizeof(int), stream));
    CUDA_TRY(launch_quantise(d_reqs, d_vps, (int)P.n, P.L.total_vp, stream));
    return VCM_OK;
}

vcm_status enqueue_launch(vcm_ctx *ctx, Slot &s, const std::vector<const Canon *> &cs,
                          const std::vector<vcm_tune> &shapes, float *const *v, uint8_t *const *color,
                          uint32_t *const *bits, vcm_stats *stats, cudaStream_t stream, bool timed = false,
                          bool adapt = true)
{
    Prepared P;
    vcm_status st = prepare_launch(ctx, s, cs, shapes, v, color, bits, stats, stream, P, adapt);
    if (st != VCM_OK)
        return st;
    return record_launch(ctx, s, P, stats, stream, timed);
}

// Same device work on the slot's stream.  A launch whose parameters equal
// those the form's graph was captured with replays the graph; one equal to
// the previous launch of the form (so likely to come again) is captured
// into the graph (updated in place when the topology allows, re-instantiated
// otherwise) and launched; any other runs directly, which costs less than a
// capture that would not be replayed.  `direct_only` launches directly.
vcm_status enqueue_graph(vcm_ctx *ctx, Slot &s, const std::vector<const Canon *> &cs,
                         const std::vector<vcm_tune> &shapes, float *const *v, uint8_t *const *color,
                         uint32_t *const *bits, vcm_stats *stats, bool one_tile, bool direct_only = false,
                         int claim_rounds = kClaimRounds, bool hold_spill = false, cudaEvent_t after = nullptr)
{
    Prepared P;
    vcm_status st = prepare_launch(ctx, s, cs, shapes, v, color, bits, stats, s.stream, P);
    if (st != VCM_OK)
        return st;
    // The graph's nodes take their arguments from the slot's buffers (the
    // descriptor upload reads the pinned arena prepare_launch just filled),
    // so a launch whose parameters all equal those of the capture replays it
    // without a new capture or update.
    const int f = one_tile ? 0 : 1;
    const auto ptr = [](const void *p) { return (unsigned long long)(uintptr_t)p; };
    const std::vector<unsigned long long> key = {
        ctx->scene_gen, P.L.off_reqs, P.L.off_tiles, P.L.off_vps, P.L.off_coords, P.L.bytes,
        (unsigned long long)P.L.total_tiles, (unsigned long long)P.L.total_vp, (unsigned long long)P.box_cap,
        (unsigned long long)P.blocks, P.n, (unsigned long long)P.extra, (unsigned long long)P.any_bits,
        (unsigned long long)P.tile_check, ptr(s.d_desc), ptr(s.h_desc), ptr(s.d_work), ptr(s.d_spill),
        ptr(s.d_spill_busy), ptr(stats)};
    direct_only = direct_only || after != nullptr;   // a graph holds no wait on another stream's event
    s.chained = false;
    if (!direct_only && s.exec[f] && s.key[f] == key) {
        CUDA_TRY(cudaGraphLaunch(s.exec[f], s.stream));
        CUDA_TRY(cudaEventRecord(s.desc_copied, s.stream));
        return VCM_OK;
    }
    if (direct_only || s.last_key[f] != key) {
        if (!direct_only)
            s.last_key[f] = key;
        return record_launch(ctx, s, P, stats, s.stream, false, false, one_tile, claim_rounds, hold_spill, after);
    }
    s.key[f].clear();
    CUDA_TRY(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeRelaxed));
    // one_tile: one block per tile, so launches of other slots interleave
    st = record_launch(ctx, s, P, stats, s.stream, false, true, one_tile);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s.stream, &g);
    if (st != VCM_OK) {
        if (g)
            cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess)
        return fail(VCM_E_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    if (s.exec[f]) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(s.exec[f], g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(s.exec[f]);
            s.exec[f] = nullptr;
        }
    }
    if (!s.exec[f]) {
        e = cudaGraphInstantiate(&s.exec[f], g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            s.exec[f] = nullptr;
            return fail(VCM_E_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
    }
    if (s.graph[f])
        cudaGraphDestroy(s.graph[f]);
    s.graph[f] = g;
    s.key[f] = key;
    CUDA_TRY(cudaGraphLaunch(s.exec[f], s.stream));
    CUDA_TRY(cudaEventRecord(s.desc_copied, s.stream));
    return VCM_OK;
}

// ---------------------------------------------------------------------------
// scene
// ---------------------------------------------------------------------------

void free_scene(vcm_ctx *ctx)
{
    cudaFree(ctx->d_lo);
    cudaFree(ctx->d_hi);
    ctx->d_lo = ctx->d_hi = nullptr;
    for (auto &p : ctx->d_perm) {
        cudaFree(p);
        p = nullptr;
    }
    cudaFree(ctx->d_cell_start);
    cudaFree(ctx->d_cell_of);
    cudaFree(ctx->d_count);
    cudaFree(ctx->d_cursor);
    cudaFree(ctx->d_order);
    cudaFree(ctx->d_cell_lo);
    cudaFree(ctx->d_cell_hi);
    cudaFree(ctx->d_overhang);
    cudaFree(ctx->d_recolor_list);
    cudaFree(ctx->d_recolor_n);
    ctx->d_cell_start = ctx->d_cell_of = ctx->d_count = ctx->d_cursor = ctx->d_order = nullptr;
    ctx->d_cell_lo = ctx->d_cell_hi = nullptr;
    ctx->d_overhang = nullptr;
    ctx->lo_cap = ctx->idx_box_cap = ctx->idx_cell_cap = 0;
    ctx->built = false;
}

bool scheduler_idle(vcm_ctx *ctx) { return ctx->queue.empty() && ctx->running_groups == 0; }

// ---------------------------------------------------------------------------
// scheduler
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// occlusion bits kept for recolouring (VCM_CACHE_BITS)
// ---------------------------------------------------------------------------

// The canonical geometry that fixes a request's occlusion bits: the
// normal's axis, side and coordinate, the patch centres and the viewpoint
// grid.  Field of view, gaze, sides, strictness and colours are left out.
std::vector<float> cache_key(const Canon &c)
{
    std::vector<float> k = {(float)c.dims, (float)c.au, (float)c.an, (float)c.aw, c.sn, c.p_n,
                            (float)c.nu, (float)c.nw, (float)c.nx, (float)c.ny, (float)c.nl};
    for (const std::vector<float> *v : {&c.u_coord, &c.w_coord, &c.x_coord, &c.y_coord, &c.z_coord})
        k.insert(k.end(), v->begin(), v->end());
    return k;
}

size_t bits_bytes(const Canon &c) { return (size_t)c.n_vp * c.words * sizeof(uint32_t); }

// A request the recolour kernels can serve (their viewpoint list is int).
bool cacheable(const Canon &c) { return !(c.flags & VCM_VIEWER) && c.n_vp <= (long long)INT32_MAX; }

std::shared_ptr<CacheEntry> cache_find(vcm_ctx *ctx, const Canon &c, bool ready_only)
{
    if (ctx->cache.empty() || !cacheable(c))
        return nullptr;
    const std::vector<float> key = cache_key(c);
    for (auto &e : ctx->cache)
        if (e->scene_gen == ctx->scene_gen && (e->ready || !ready_only) && e->key == key)
            return e;
    return nullptr;
}

void cache_drop(vcm_ctx *ctx, const std::shared_ptr<CacheEntry> &e)
{
    auto it = std::find(ctx->cache.begin(), ctx->cache.end(), e);
    if (it == ctx->cache.end())
        return;
    if (e->d_bits)
        cudaFreeAsync(e->d_bits, ctx->aux);
    e->d_bits = nullptr;
    ctx->cache_bytes -= e->bytes;
    ctx->cache.erase(it);
}

// Drop the least recently used entry that no launch uses; false if none.
bool cache_evict_one(vcm_ctx *ctx)
{
    std::shared_ptr<CacheEntry> victim;
    for (auto &e : ctx->cache)
        if (e->users == 0 && (!victim || e->last_use < victim->last_use))
            victim = e;
    if (!victim)
        return false;
    cache_drop(ctx, victim);
    return true;
}

// Drop every entry no launch uses (all of them when nothing runs).
void cache_clear(vcm_ctx *ctx)
{
    while (cache_evict_one(ctx)) {
    }
}

constexpr size_t kLatencyRing = 4096;

// A completed request: its latency into the ring (when it succeeded) and,
// with the request log on, its metric line (called with ctx->mu held).
void note_completion(vcm_ctx *ctx, const Ticket &t, std::string &lines)
{
    const double lat = std::chrono::duration<double, std::milli>(t.t_done - t.t_submit).count();
    if (t.state == T_DONE) {
        if (ctx->lat_ring.size() < kLatencyRing)
            ctx->lat_ring.push_back(lat);
        else
            ctx->lat_ring[ctx->lat_done % kLatencyRing] = lat;
        ctx->lat_done++;
    }
    if (!ctx->log_on.load(std::memory_order_relaxed))
        return;
    const Canon &c = t.canon;
    const vcm_stats z{};
    const vcm_stats &st = (t.h_stats && t.state == T_DONE) ? *t.h_stats : z;
    char buf[768];
    std::snprintf(buf, sizeof buf,
                  "{\"ticket\": %llu, \"status\": %d, \"latency_ms\": %.6f, \"queue_ms\": %.6f, "
                  "\"launch_ms\": %.6f, \"device_ms\": %.6f, \"chain_ms\": %.6f, \"group_size\": %u, "
                  "\"launch_form\": %u, \"viewpoints\": %lld, \"patches\": %d, \"segments\": %llu, "
                  "\"slab_tests\": %llu, \"corner_tests\": %llu, \"rechecked\": %llu, \"edge_cells\": %u, "
                  "\"shortcut_viewpoints\": %llu, \"shared_viewpoints\": %llu, \"v_ref\": %.9g}\n",
                  (unsigned long long)t.id, t.state == T_DONE ? 0 : (int)t.err, lat,
                  std::chrono::duration<double, std::milli>(t.t_launch - t.t_submit).count(), t.launch_ms,
                  t.device_ms, t.chain_ms, t.group_size, t.form, (long long)c.n_vp, c.P,
                  (unsigned long long)c.n_vp * (unsigned long long)c.P, st.slab_tests, st.corner_tests,
                  st.rechecked, st.edge_cells, st.shortcut_viewpoints, st.shared_viewpoints, (double)st.v_ref);
    lines += buf;
}


// Completion of a slot's launches.  CUDA host callbacks are not used: a
// callback that takes the context lock can deadlock against a thread that
// holds the lock inside a call that implicitly synchronises the device
// (cudaMallocHost, cudaFree).  This thread waits on the slot's event with no
// lock held and only then takes the lock.
void slot_waiter(vcm_ctx *ctx, Slot *s)
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    for (;;) {
        ctx->cv.wait(lk, [&] { return s->posted || ctx->stop; });
        if (!s->posted)
            return;   // stopping with nothing in flight
        std::vector<std::shared_ptr<Ticket>> group;
        group.swap(s->inflight);
        s->posted = false;
        cudaEvent_t ev = s->done;
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(ev);
        const auto now = std::chrono::steady_clock::now();
        float dev_ms = 0.f, chain_ms = 0.f;
        if (e == cudaSuccess && cudaEventElapsedTime(&dev_ms, s->t0, s->t1) != cudaSuccess) {
            cudaGetLastError();
            dev_ms = 0.f;
        }
        if (e == cudaSuccess && s->chained && cudaEventElapsedTime(&chain_ms, s->t0, s->t_chain) != cudaSuccess) {
            cudaGetLastError();
            chain_ms = 0.f;
        }
        lk.lock();
        for (auto &t : group) {
            t->device_ms = dev_ms;
            t->chain_ms = chain_ms;
            const uint32_t derr = t->h_stats ? t->h_stats->error : 0u;
            if (e != cudaSuccess) {
                t->state = T_ERROR;
                t->err = VCM_E_CUDA;
                t->msg = std::string("launch failed: ") + cudaGetErrorString(e);
            } else if (derr == VCM_DEVERR_SPILL_WAIT) {
                t->state = T_ERROR;
                t->err = VCM_E_TIMEOUT;
                t->msg = "a bounded device-side wait for a spill region gave up; the result is incomplete";
            } else if (derr) {
                t->state = T_ERROR;
                t->err = VCM_E_CUDA;
                t->msg = "device-side bounds check failed (error " + std::to_string(derr) + ")";
            } else {
                t->state = T_DONE;
            }
            t->t_done = now;
            if (t->cache_fill) {   // the bits are there once the launch has run cleanly
                auto e = t->cache_fill;
                e->users--;
                e->ready = t->state == T_DONE;
                if (!e->ready && e->users == 0)
                    cache_drop(ctx, e);
                t->cache_fill.reset();
            }
            if (t->cache_hit) {
                t->cache_hit->users--;
                t->cache_hit.reset();
            }
        }
        s->busy = false;
        ctx->running_groups--;
        ctx->cv.notify_all();
        std::string lines;
        for (auto &t : group)
            note_completion(ctx, *t, lines);
        if (!lines.empty()) {
            lk.unlock();
            {
                std::lock_guard<std::mutex> g(ctx->log_mu);
                if (ctx->req_log) {
                    fputs(lines.c_str(), ctx->req_log);
                    fflush(ctx->req_log);
                }
            }
            lk.lock();
        }
    }
}

void release_buffers(vcm_ctx *ctx, Ticket &t)
{
    if (t.d_v)
        cudaFreeAsync(t.d_v, ctx->aux);
    t.d_v = nullptr;
    t.d_color = nullptr;
    t.d_bits = nullptr;
    ctx->pinned.put(t.h_v);
    t.h_v = nullptr;
    t.h_color = nullptr;
    t.h_bits = nullptr;
    t.h_stats = nullptr;
    if (t.bytes) {
        ctx->used -= t.bytes;
        t.bytes = 0;
    }
}

// Allocate one request's device and pinned buffers (one block each).
// Layout: v (floats) | color | bits | stats.
bool alloc_buffers(vcm_ctx *ctx, Ticket &t, cudaStream_t stream)
{
    if (ctx->inject_alloc > 0) {   // vcm_inject: this allocation fails
        --ctx->inject_alloc;
        return false;
    }
    const Canon &c = t.canon;
    const size_t n = (size_t)c.n_vp;
    const size_t off_color = align_up(n * 4, 256);
    const size_t off_bits = align_up(off_color + n, 256);
    const size_t bits_bytes = (c.flags & VCM_EMIT_BITS) ? n * c.words * 4 : 0;
    const size_t off_stats = align_up(off_bits + bits_bytes, 256);
    const size_t total = off_stats + sizeof(vcm_stats);
    char *d = nullptr;
    if (cudaMallocAsync((void **)&d, total, stream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    char *h = static_cast<char *>(ctx->pinned.get(total));
    if (!h) {
        cudaFreeAsync(d, stream);
        return false;
    }
    t.d_v = reinterpret_cast<float *>(d);
    t.d_color = reinterpret_cast<uint8_t *>(d + off_color);
    t.d_bits = bits_bytes ? reinterpret_cast<uint32_t *>(d + off_bits) : nullptr;
    t.h_v = reinterpret_cast<float *>(h);
    t.h_color = reinterpret_cast<uint8_t *>(h + off_color);
    t.h_bits = bits_bytes ? reinterpret_cast<uint32_t *>(h + off_bits) : nullptr;
    t.h_stats = reinterpret_cast<vcm_stats *>(h + off_stats);
    return true;
}

// Launch one admitted group on its slot (called with ctx->mu held).
void launch_group(vcm_ctx *ctx, Slot &s, std::vector<std::shared_ptr<Ticket>> &group)
{
    Range range("vcm launch group");
    std::vector<const Canon *> cs;
    std::vector<vcm_tune> shapes;
    std::vector<float *> v;
    std::vector<uint8_t *> col;
    std::vector<uint32_t *> bits;
    // a request that fills cached bits emits them into the cache's buffer
    std::vector<Canon> filling(group.size());
    for (size_t i = 0; i < group.size(); ++i) {
        auto &t = group[i];
        if (t->cache_fill) {
            filling[i] = t->canon;
            filling[i].flags |= VCM_EMIT_BITS;
            cs.push_back(&filling[i]);
            bits.push_back(t->cache_fill->d_bits);
        } else {
            cs.push_back(&t->canon);
            bits.push_back(t->d_bits);
        }
        shapes.push_back(t->shape);
        v.push_back(t->d_v);
        col.push_back(t->d_color);
    }
    vcm_status st = ensure_slot(ctx, s, 0, group.size(), 1, s.stream);
    // Every group gets the persistent grid and its chunk pass, and at most
    // as many groups as there are slots are in flight (two by default).  A
    // group launched while another is in flight uploads its descriptors and
    // clears its counters at once, then its stream waits for the other's
    // kernels before its tile kernel: the device runs the launches' kernels
    // back to back with no gap for the host, the result copies of one
    // overlap the kernels of the next, and requests that arrive meanwhile
    // are batched into the launch after it.  Persistent grids that ran side
    // by side starved each other's chunk pass (a request of 3.4 ms took
    // 12 ms), and one block per tile beside other launches made a large
    // request 2-3 times slower than alone.  One block per tile remains for
    // the spill-claim fault injection.
    const bool inject = ctx->inject_spill > 0;
    if (inject)
        --ctx->inject_spill;
    const bool one_tile = inject;
    cudaEvent_t after = nullptr;
    if (ctx->last_launched && ctx->last_launched != &s && ctx->last_launched->busy)
        after = ctx->last_launched->kernels_done;
    const auto now = std::chrono::steady_clock::now();
    for (auto &t : group) {
        t->t_launch = now;
        t->group_size = (uint32_t)group.size();
        t->form = one_tile ? VCM_FORM_ONE_TILE : VCM_FORM_PERSISTENT;
    }
    if (st == VCM_OK && cudaEventRecord(s.t0, s.stream) != cudaSuccess)
        st = fail(VCM_E_CUDA, "cudaEventRecord failed");
    if (st == VCM_OK)
        st = enqueue_graph(ctx, s, cs, shapes, v.data(), col.data(), bits.data(), s.d_stats, one_tile,
                           /*direct_only=*/inject, inject ? 8 : kClaimRounds, /*hold_spill=*/inject, after);
    if (st == VCM_OK && cudaEventRecord(s.kernels_done, s.stream) != cudaSuccess)
        st = fail(VCM_E_CUDA, "cudaEventRecord failed");
    if (st == VCM_OK) {
        for (size_t i = 0; i < group.size(); ++i) {
            Ticket &t = *group[i];
            const Canon &c = t.canon;
            if (t.cache_fill && t.d_bits)   // the caller asked for the bits too
                cudaMemcpyAsync(t.d_bits, t.cache_fill->d_bits, bits_bytes(c), cudaMemcpyDeviceToDevice, s.stream);
            cudaMemcpyAsync(t.h_v, t.d_v, (size_t)c.n_vp * 4, cudaMemcpyDeviceToHost, s.stream);
            cudaMemcpyAsync(t.h_color, t.d_color, (size_t)c.n_vp, cudaMemcpyDeviceToHost, s.stream);
            if (t.d_bits)
                cudaMemcpyAsync(t.h_bits, t.d_bits, (size_t)c.n_vp * c.words * 4, cudaMemcpyDeviceToHost,
                                s.stream);
            cudaMemcpyAsync(t.h_stats, s.d_stats + i, sizeof(vcm_stats), cudaMemcpyDeviceToHost, s.stream);
        }
        if (cudaEventRecord(s.t1, s.stream) == cudaSuccess && cudaEventRecord(s.done, s.stream) == cudaSuccess) {
            const double host_ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - now).count();
            for (auto &t : group) {
                t->state = T_RUNNING;
                t->slot = &s;
                t->launch_ms = host_ms;
            }
            s.inflight = group;
            ctx->last_launched = &s;
            s.posted = true;
            s.busy = true;
            ctx->running_groups++;
            return;
        }
        st = fail(VCM_E_CUDA, "cudaEventRecord failed");
    }
    for (auto &t : group) {
        if (t->cache_fill) {
            t->cache_fill->users--;
            cache_drop(ctx, t->cache_fill);
            t->cache_fill.reset();
        }
        t->state = T_ERROR;
        t->err = st;
        t->msg = t_err;
        t->t_done = std::chrono::steady_clock::now();
        release_buffers(ctx, *t);
    }
}

// Launch one request served from cached occlusion bits (ctx->mu held): its
// descriptor, the recolour kernels (Section IV-C: the field of view, gaze,
// sides and strictness applied to bits made earlier), colours, and the
// copies of its results, chained after the launch in flight like any other.
void launch_recolor_group(vcm_ctx *ctx, Slot &s, std::vector<std::shared_ptr<Ticket>> &group)
{
    Range range("vcm launch recolour");
    Ticket &t = *group[0];
    const std::shared_ptr<CacheEntry> e = t.cache_hit;
    Canon c = t.canon;
    c.flags &= ~(unsigned)(VCM_EMIT_BITS | VCM_CACHE_BITS);   // the bits are an input here
    const std::vector<const Canon *> cs{&c};
    const std::vector<vcm_tune> shapes{default_tune()};
    const Layout L = layout_for(cs, shapes);
    cudaEvent_t after = nullptr;
    if (ctx->last_launched && ctx->last_launched != &s && ctx->last_launched->busy)
        after = ctx->last_launched->kernels_done;
    t.t_launch = std::chrono::steady_clock::now();
    t.group_size = 1;
    t.form = VCM_FORM_RECOLOR;
    vcm_status st = ensure_slot(ctx, s, L.bytes, 1, 1, s.stream);
    auto body = [&]() -> vcm_status {
        CUDA_TRY(cudaEventSynchronize(s.desc_copied));
        float *vv[1] = {t.d_v};
        uint8_t *cc[1] = {t.d_color};
        uint32_t *bb[1] = {e->d_bits};   // read only in k_recolor
        fill_desc(s.h_desc, s.d_desc, L, cs, shapes, vv, cc, bb, s.d_stats, 256, /*blockers=*/false);
        CUDA_TRY(cudaEventRecord(s.t0, s.stream));
        CUDA_TRY(cudaMemcpyAsync(s.d_desc, s.h_desc, L.bytes, cudaMemcpyHostToDevice, s.stream));
        CUDA_TRY(cudaEventRecord(s.desc_copied, s.stream));
        CUDA_TRY(cudaMemsetAsync(s.d_stats, 0, sizeof(vcm_stats), s.stream));
        s.chained = false;
        if (after) {
            CUDA_TRY(cudaStreamWaitEvent(s.stream, after, 0));
            CUDA_TRY(cudaEventRecord(s.t_chain, s.stream));
            s.chained = true;
        }
        const DevRequest *d_reqs = reinterpret_cast<const DevRequest *>(s.d_desc + L.off_reqs);
        const long long *d_vps = reinterpret_cast<const long long *>(s.d_desc + L.off_vps);
        int *list = nullptr;   // the viewpoints that need a measure, and their count
        CUDA_TRY(cudaMallocAsync((void **)&list, sizeof(int) * ((size_t)c.n_vp + 1), s.stream));
        const cudaError_t le = launch_recolor(d_reqs, c.n_vp, ctx->sm_count, list, list + c.n_vp, s.stream);
        cudaFreeAsync(list, s.stream);
        CUDA_TRY(le);
        CUDA_TRY(launch_quantise(d_reqs, d_vps, 1, c.n_vp, s.stream));
        CUDA_TRY(cudaEventRecord(s.kernels_done, s.stream));
        CUDA_TRY(cudaMemcpyAsync(t.h_v, t.d_v, (size_t)c.n_vp * 4, cudaMemcpyDeviceToHost, s.stream));
        CUDA_TRY(cudaMemcpyAsync(t.h_color, t.d_color, (size_t)c.n_vp, cudaMemcpyDeviceToHost, s.stream));
        if (t.d_bits) {
            CUDA_TRY(cudaMemcpyAsync(t.d_bits, e->d_bits, bits_bytes(c), cudaMemcpyDeviceToDevice, s.stream));
            CUDA_TRY(cudaMemcpyAsync(t.h_bits, e->d_bits, bits_bytes(c), cudaMemcpyDeviceToHost, s.stream));
        }
        CUDA_TRY(cudaMemcpyAsync(t.h_stats, s.d_stats, sizeof(vcm_stats), cudaMemcpyDeviceToHost, s.stream));
        CUDA_TRY(cudaEventRecord(s.t1, s.stream));
        CUDA_TRY(cudaEventRecord(s.done, s.stream));
        return VCM_OK;
    };
    if (st == VCM_OK)
        st = body();
    if (st == VCM_OK) {
        t.launch_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t.t_launch).count();
        t.state = T_RUNNING;
        t.slot = &s;
        s.inflight = group;
        ctx->last_launched = &s;
        s.posted = true;
        s.busy = true;
        ctx->running_groups++;
        return;
    }
    e->users--;
    t.cache_hit.reset();
    t.state = T_ERROR;
    t.err = st;
    t.msg = t_err;
    t.t_done = std::chrono::steady_clock::now();
    release_buffers(ctx, t);
}

enum SchedStep { STEP_WAIT, STEP_LAUNCHED, STEP_PROGRESS };

// Free the scratch of an idle scheduler slot (and the graphs that use it);
// the next launch on the slot allocates it again.  Only with nothing in
// flight on the slot.
void release_slot_scratch(vcm_ctx *ctx, Slot &s)
{
    for (int f = 0; f < 2; ++f) {
        if (s.exec[f]) cudaGraphExecDestroy(s.exec[f]);
        if (s.graph[f]) cudaGraphDestroy(s.graph[f]);
        s.exec[f] = nullptr;
        s.graph[f] = nullptr;
        s.key[f].clear();
        s.last_key[f].clear();
    }
    cudaStreamSynchronize(s.stream);
    if (s.d_desc) cudaFree(s.d_desc);
    if (s.h_desc) cudaFreeHost(s.h_desc);
    if (s.d_work) cudaFree(s.d_work);
    if (s.d_spill) cudaFree(s.d_spill);
    if (s.d_spill_busy) cudaFree(s.d_spill_busy);
    if (s.d_stats) cudaFree(s.d_stats);
    s.d_desc = s.h_desc = nullptr;
    s.d_work = s.d_spill = s.d_spill_busy = nullptr;
    s.d_stats = nullptr;
    s.desc_cap = s.spill_cap = s.spill_busy_cap = s.stats_cap = 0;
    if (s.scheduler)
        ctx->scratch -= s.scratch;
    s.scratch = 0;
}

// One scheduling decision (ctx->mu held): admit a batch from the head of the
// queue onto a free slot and launch it.  Called by the scheduler thread and,
// once, inline by vcm_submit so that a request that can start at once does
// not wait for a thread hand-off.
//
// Admission charges the budget with the result buffers of admitted requests
// and the scratch of the slots, including what the chosen slot still has to
// allocate for its first launch.
SchedStep schedule_once(vcm_ctx *ctx)
{
    if (ctx->queue.empty())
        return STEP_WAIT;
    // Small work goes to a free high-priority slot (its blocks start as
    // soon as blocks of a running big launch finish); big work to a
    // low-priority one.  Either may use the other kind when that is all
    // that is free.
    double head_work = 0.0;
    size_t head_need = 0;
    for (auto &t : ctx->queue.front()) {
        head_work += (double)t->canon.n_vp * t->canon.P;
        head_need += t->canon.out_bytes() + 1024;
    }
    const bool small = head_work <= kSmallWork;
    const size_t scratch_need = slot_scratch_need(ctx);
    auto growth = [&](const Slot *s) { return scratch_need > s->scratch ? scratch_need - s->scratch : 0; };
    const size_t held = ctx->used + ctx->scratch + ctx->cache_bytes;   // charged against the budget
    Slot *free_slot = nullptr;
    bool any_free = false;
    for (int trimmed = 0; trimmed < 2 && !free_slot; ++trimmed) {
        // free slots by preference (matching priority, then any); the first
        // whose scratch growth and the head's results fit the budget
        for (int pass = 0; pass < 2 && !free_slot; ++pass)
            for (auto &s : ctx->slots)
                if (!s->busy && (pass == 1 || s->high_priority == small)) {
                    any_free = true;
                    if (held + growth(s.get()) + head_need <= ctx->budget) {
                        free_slot = s.get();
                        break;
                    }
                }
        if (free_slot || !any_free || trimmed || ctx->running_groups > 0)
            break;
        // Nothing runs and the head does not fit: give back the scratch of
        // idle slots, keeping one slot's, and try again.
        Slot *keep = nullptr;
        for (auto &s : ctx->slots)
            if (!keep || s->scratch > keep->scratch)
                keep = s.get();
        for (auto &s : ctx->slots)
            if (s.get() != keep && s->scratch)
                release_slot_scratch(ctx, *s);
    }
    if (!free_slot)
        return STEP_WAIT;   // finished results still hold memory until released
    // admit groups from the front of the queue while memory allows
    std::vector<std::shared_ptr<Ticket>> batch;
    bool alloc_failed = false, recolour = false;
    double batch_work = 0.0;
    const size_t slot_growth = growth(free_slot);
    while (!ctx->queue.empty()) {
        auto &grp = ctx->queue.front();
        // a request whose bits are cached runs alone, as a recolour
        std::shared_ptr<CacheEntry> hit = grp.size() == 1 ? cache_find(ctx, grp[0]->canon, true) : nullptr;
        if (hit && !batch.empty())
            break;
        size_t need = 0, fill = 0;
        double work = 0.0;
        for (auto &t : grp) {
            need += t->canon.out_bytes() + 1024;
            work += (double)t->canon.n_vp * t->canon.P;
            if (!hit && (t->canon.flags & VCM_CACHE_BITS) && cacheable(t->canon) && !cache_find(ctx, t->canon, false))
                fill += bits_bytes(t->canon);
        }
        if (hit)
            need += sizeof(int) * ((size_t)grp[0]->canon.n_vp + 1);   // the recolour's viewpoint list
        if (!batch.empty() && batch.size() + grp.size() > ctx->max_batch)
            break;
        // a batch completes as a whole: keep small requests out of big batches
        if (!batch.empty() && batch_work + work > kBatchWork)
            break;
        if (ctx->used + ctx->scratch + ctx->cache_bytes + slot_growth + need + fill > ctx->budget) {
            // cached bits nobody uses give way to admitted work
            if (cache_evict_one(ctx))
                continue;
            break;
        }
        bool ok = true;
        for (auto &t : grp) {
            if (!alloc_buffers(ctx, *t, free_slot->stream)) {
                ok = false;
                break;
            }
            t->bytes = t->canon.out_bytes() + 1024;
            ctx->used += t->bytes;
        }
        if (!ok) {
            for (auto &t : grp)
                release_buffers(ctx, *t);
            alloc_failed = true;
            break;
        }
        for (auto &t : grp) {
            if (hit) {
                t->cache_hit = hit;
                hit->users++;
                hit->last_use = ++ctx->cache_clock;
            } else if ((t->canon.flags & VCM_CACHE_BITS) && cacheable(t->canon) && !cache_find(ctx, t->canon, false)) {
                // this launch fills the cache (a failed allocation only skips caching)
                auto e = std::make_shared<CacheEntry>();
                e->key = cache_key(t->canon);
                e->scene_gen = ctx->scene_gen;
                e->bytes = bits_bytes(t->canon);
                if (cudaMallocAsync((void **)&e->d_bits, e->bytes, free_slot->stream) == cudaSuccess) {
                    e->users = 1;
                    e->last_use = ++ctx->cache_clock;
                    ctx->cache.push_back(e);
                    ctx->cache_bytes += e->bytes;
                    t->cache_fill = e;
                } else {
                    cudaGetLastError();
                }
            }
            batch.push_back(t);
        }
        batch_work += work;
        ctx->queue.pop_front();
        if (hit) {
            recolour = true;
            break;
        }
    }
    if (batch.empty()) {
        // Only a device allocation that fails with nothing in flight is
        // final; otherwise wait for memory to free up.
        if (alloc_failed && ctx->running_groups == 0) {
            auto grp = ctx->queue.front();
            ctx->queue.pop_front();
            for (auto &t : grp) {
                t->state = T_ERROR;
                t->err = VCM_E_NOMEM;
                t->msg = "request does not fit in device memory";
                t->t_done = std::chrono::steady_clock::now();
            }
            return STEP_PROGRESS;
        }
        return STEP_WAIT;
    }
    if (recolour)
        launch_recolor_group(ctx, *free_slot, batch);
    else
        launch_group(ctx, *free_slot, batch);
    return STEP_LAUNCHED;
}

void scheduler_loop(vcm_ctx *ctx)
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (!ctx->stop) {
        const SchedStep st = schedule_once(ctx);
        if (st == STEP_WAIT)
            ctx->cv.wait(lk);
        else
            ctx->cv.notify_all();
    }
}

vcm_status start_scheduler(vcm_ctx *ctx, uint32_t n_slots)
{
    int prio_low = 0, prio_high = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    for (uint32_t i = 0; i < n_slots; ++i) {
        auto s = std::make_unique<Slot>();
        // the first half of the slots run small batches at high priority
        s->high_priority = n_slots > 1 && i < n_slots / 2;
        CUDA_TRY(cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking,
                                              s->high_priority ? prio_high : prio_low));
        CUDA_TRY(cudaEventCreateWithFlags(&s->desc_copied, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreate(&s->t0));
        CUDA_TRY(cudaEventCreate(&s->t1));
        CUDA_TRY(cudaEventCreateWithFlags(&s->kernels_done, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreate(&s->t_chain));
        s->scheduler = true;
        ctx->slots.push_back(std::move(s));
    }
    ctx->stop = false;
    for (auto &s : ctx->slots)
        s->waiter = std::thread(slot_waiter, ctx, s.get());
    ctx->worker = std::thread(scheduler_loop, ctx);
    return VCM_OK;
}

void stop_scheduler(vcm_ctx *ctx)
{
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv.notify_all();
    if (ctx->worker.joinable())
        ctx->worker.join();
    for (auto &s : ctx->slots) {
        if (s->waiter.joinable())
            s->waiter.join();   // finishes any posted group first
        if (s->stream)
            cudaStreamSynchronize(s->stream);
    }
}

void destroy_slot(Slot &s)
{
    for (int f = 0; f < 2; ++f) {
        if (s.exec[f]) cudaGraphExecDestroy(s.exec[f]);
        if (s.graph[f]) cudaGraphDestroy(s.graph[f]);
    }
    if (s.d_desc) cudaFree(s.d_desc);
    if (s.h_desc) cudaFreeHost(s.h_desc);
    if (s.d_work) cudaFree(s.d_work);
    if (s.d_spill) cudaFree(s.d_spill);
    if (s.d_spill_busy) cudaFree(s.d_spill_busy);
    if (s.d_stats) cudaFree(s.d_stats);
    if (s.desc_copied) cudaEventDestroy(s.desc_copied);
    if (s.done) cudaEventDestroy(s.done);
    if (s.t0) cudaEventDestroy(s.t0);
    if (s.t1) cudaEventDestroy(s.t1);
    if (s.kernels_done) cudaEventDestroy(s.kernels_done);
    if (s.t_chain) cudaEventDestroy(s.t_chain);
    s.t0 = s.t1 = s.kernels_done = s.t_chain = nullptr;
    if (s.stream) cudaStreamDestroy(s.stream);
    s.inflight.clear();
    s.stream = nullptr;
    s.desc_copied = s.done = nullptr;
    s.d_desc = s.h_desc = nullptr;
    s.desc_cap = 0;
    s.d_work = s.d_spill = s.d_spill_busy = nullptr;
    s.spill_cap = s.spill_busy_cap = 0;
    s.d_stats = nullptr;
    s.stats_cap = 0;
    s.scratch = 0;
    s.busy = s.posted = false;
    s.graph[0] = s.graph[1] = nullptr;
    s.exec[0] = s.exec[1] = nullptr;
}

vcm_status validate_ctx(vcm_ctx *ctx)
{
    if (!ctx)
        return fail(VCM_E_ARG, "context is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess)
        return fail(VCM_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return VCM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

vcm_status vcm_ctx_create(int device, size_t mem_budget_bytes, vcm_ctx **out)
{
    try {
        if (!out)
            return fail(VCM_E_ARG, "out is NULL");
        *out = nullptr;
        int n = 0;
        cudaError_t e = cudaGetDeviceCount(&n);
        if (e != cudaSuccess || n == 0)
            return fail(VCM_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
        if (device < 0 || device >= n)
            return fail(VCM_E_ARG, "device %d out of range (%d devices)", device, n);
        CUDA_TRY(cudaSetDevice(device));
        CUDA_TRY(init_device());
        auto ctx = std::make_unique<vcm_ctx>();
        ctx->device = device;
        CUDA_TRY(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
        ctx->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)64 << 30;
        for (auto &t : ctx->tune)
            t = default_tune();
        CUDA_TRY(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&ctx->direct.desc_copied, cudaEventDisableTiming));
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        vcm_status st = start_scheduler(ctx.get(), 2);
        if (st != VCM_OK)
            return st;
        *out = ctx.release();
        return VCM_OK;
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_ctx_create: %s", ex.what());
    }
}

void vcm_ctx_destroy(vcm_ctx *ctx)
{
    if (!ctx)
        return;
    cudaSetDevice(ctx->device);
    stop_scheduler(ctx);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        for (auto &kv : ctx->tickets)
            release_buffers(ctx, *kv.second);
        ctx->tickets.clear();
        for (auto &e : ctx->cache)
            e->users = 0;   // nothing runs any more
        cache_clear(ctx);
    }
    cudaStreamSynchronize(ctx->aux);
    for (auto &s : ctx->slots)
        destroy_slot(*s);
    destroy_slot(ctx->direct);
    free_scene(ctx);
    if (ctx->aux)
        cudaStreamDestroy(ctx->aux);
    if (ctx->req_log)
        fclose(ctx->req_log);
    delete ctx;
}

const char *vcm_last_error(vcm_ctx *)
{
    return t_err.c_str();
}

vcm_status vcm_scene_load_mem(vcm_ctx *ctx, const float *lo, const float *hi, uint32_t n_boxes, int32_t dims)
{
    Range range("vcm_scene_load_mem");
    try {
        vcm_status st = validate_ctx(ctx);
        if (st != VCM_OK)
            return st;
        if (dims != 2 && dims != 3)
            return fail(VCM_E_ARG, "dims must be 2 or 3");
        if (n_boxes > 0 && (!lo || !hi))
            return fail(VCM_E_ARG, "lo/hi are NULL");
        if (n_boxes > (1u << 26))
            return fail(VCM_E_ARG, "too many boxes (%u)", n_boxes);
        std::vector<float> L((size_t)n_boxes * 3, 0.f), H((size_t)n_boxes * 3, 0.f);
        for (uint32_t i = 0; i < n_boxes; ++i)
            for (int k = 0; k < dims; ++k) {
                const float a = lo[(size_t)i * dims + k], b = hi[(size_t)i * dims + k];
                int64_t ua, ub;
                if (!to_units(a, ua) || !to_units(b, ub))
                    return fail(VCM_E_ARG, "box %u coordinate %d is not a finite lattice value within 16384 m", i, k);
                if (ua > ub)
                    return fail(VCM_E_ARG, "box %u has lo > hi on axis %d", i, k);
                L[(size_t)i * 3 + k] = a;
                H[(size_t)i * 3 + k] = b;
            }
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!scheduler_idle(ctx))
            return fail(VCM_E_STATE, "requests are still queued or running");
        // work still reading the old scene must finish before it is replaced
        CUDA_TRY(cudaDeviceSynchronize());
        cache_clear(ctx);   // cached bits belong to the old scene
        ctx->built = false;
        ctx->dims = dims;
        ctx->n_boxes = n_boxes;
        ctx->h_lo.swap(L);
        ctx->h_hi.swap(H);
        const size_t nb = std::max<uint32_t>(n_boxes, 1);
        if (nb > ctx->lo_cap) {   // buffers are kept and reused while large enough
            cudaFree(ctx->d_lo);
            cudaFree(ctx->d_hi);
            ctx->d_lo = ctx->d_hi = nullptr;
            ctx->lo_cap = 0;
            CUDA_TRY(cudaMalloc(&ctx->d_lo, nb * 3 * sizeof(float)));
            CUDA_TRY(cudaMalloc(&ctx->d_hi, nb * 3 * sizeof(float)));
            ctx->lo_cap = nb;
        }
        if (n_boxes) {
            CUDA_TRY(cudaMemcpy(ctx->d_lo, ctx->h_lo.data(), (size_t)n_boxes * 12, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(ctx->d_hi, ctx->h_hi.data(), (size_t)n_boxes * 12, cudaMemcpyHostToDevice));
        }
        return VCM_OK;
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_scene_load_mem: %s", ex.what());
    }
}

vcm_status vcm_scene_load(vcm_ctx *ctx, const char *path)
{
    if (!path)
        return fail(VCM_E_ARG, "path is NULL");
    FILE *f = fopen(path, "rb");
    if (!f)
        return fail(VCM_E_IO, "cannot open %s", path);
    char magic[4];
    uint32_t version = 0, n = 0;
    int32_t dims = 0;
    bool ok = fread(magic, 1, 4, f) == 4 && std::memcmp(magic, "VCMS", 4) == 0 &&
              fread(&version, 4, 1, f) == 1 && version == 1 && fread(&dims, 4, 1, f) == 1 &&
              fread(&n, 4, 1, f) == 1 && (dims == 2 || dims == 3) && n <= (1u << 26);
    std::vector<float> lo, hi;
    if (ok) {
        lo.resize((size_t)n * dims);
        hi.resize((size_t)n * dims);
        ok = fread(lo.data(), sizeof(float), lo.size(), f) == lo.size() &&
             fread(hi.data(), sizeof(float), hi.size(), f) == hi.size();
        char extra;
        if (ok && fread(&extra, 1, 1, f) == 1)
            ok = false;   // trailing bytes
    }
    fclose(f);
    if (!ok)
        return fail(VCM_E_IO, "%s is not a valid scene file", path);
    return vcm_scene_load_mem(ctx, lo.data(), hi.data(), n, dims);
}

vcm_status vcm_scene_save(vcm_ctx *ctx, const char *path)
{
    if (!ctx || !path)
        return fail(VCM_E_ARG, "NULL argument");
    if (ctx->dims == 0)
        return fail(VCM_E_STATE, "no scene loaded");
    FILE *f = fopen(path, "wb");
    if (!f)
        return fail(VCM_E_IO, "cannot write %s", path);
    const uint32_t version = 1, n = ctx->n_boxes;
    const int32_t dims = ctx->dims;
    bool ok = fwrite("VCMS", 1, 4, f) == 4 && fwrite(&version, 4, 1, f) == 1 && fwrite(&dims, 4, 1, f) == 1 &&
              fwrite(&n, 4, 1, f) == 1;
    for (int pass = 0; pass < 2 && ok; ++pass) {
        const std::vector<float> &src = pass ? ctx->h_hi : ctx->h_lo;
        for (uint32_t i = 0; i < n && ok; ++i)
            ok = fwrite(&src[(size_t)i * 3], sizeof(float), dims, f) == (size_t)dims;
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? VCM_OK : fail(VCM_E_IO, "write to %s failed", path);
}

vcm_status vcm_build(vcm_ctx *ctx, float grid_cell_m)
{
    Range range("vcm_build");
    try {
        vcm_status st = validate_ctx(ctx);
        if (st != VCM_OK)
            return st;
        if (ctx->dims == 0)
            return fail(VCM_E_STATE, "no scene loaded");
        if (!std::isfinite(grid_cell_m) || grid_cell_m < 0.f)
            return fail(VCM_E_ARG, "grid_cell_m must be >= 0");
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!scheduler_idle(ctx))
            return fail(VCM_E_STATE, "requests are still queued or running");
        const uint32_t n = ctx->n_boxes;
        double x0 = 0, x1 = 1, y0 = 0, y1 = 1, side = 0;
        if (n) {
            x0 = y0 = 1e30;
            x1 = y1 = -1e30;
            for (uint32_t i = 0; i < n; ++i) {
                x0 = std::min<double>(x0, ctx->h_lo[3 * i]);
                y0 = std::min<double>(y0, ctx->h_lo[3 * i + 1]);
                x1 = std::max<double>(x1, ctx->h_hi[3 * i]);
                y1 = std::max<double>(y1, ctx->h_hi[3 * i + 1]);
                side += std::sqrt(std::max(0.0, (double)(ctx->h_hi[3 * i] - ctx->h_lo[3 * i]) *
                                                    (ctx->h_hi[3 * i + 1] - ctx->h_lo[3 * i + 1])));
            }
            side /= n;
        }
        const double w = std::max(x1 - x0, 1.0), h = std::max(y1 - y0, 1.0);
        double cell = grid_cell_m;
        if (cell <= 0.0)
            cell = std::max({side, std::sqrt(w * h / std::max<uint32_t>(n, 1)) * 1.5, 1.0});
        // keep the grid at most 4M cells
        while ((w / cell + 1) * (h / cell + 1) > 4.0e6)
            cell *= 1.5;
        const int gnx = (int)std::ceil(w / cell) + 1, gny = (int)std::ceil(h / cell) + 1;
        const int n_cells = gnx * gny;
        // work still reading the old index must finish before it is rebuilt
        CUDA_TRY(cudaDeviceSynchronize());
        cache_clear(ctx);   // cached bits belong to the old index's scene
        ctx->built = false;
        const size_t nb = std::max<uint32_t>(n, 1);
        if (nb > ctx->idx_box_cap) {   // index buffers are reused while large enough
            for (auto &p : ctx->d_perm) {
                cudaFree(p);
                p = nullptr;
            }
            cudaFree(ctx->d_cell_of);
            cudaFree(ctx->d_order);
            ctx->d_cell_of = ctx->d_order = nullptr;
            ctx->idx_box_cap = 0;
            for (auto &p : ctx->d_perm)
                CUDA_TRY(cudaMalloc(&p, nb * 2 * sizeof(float4)));
            CUDA_TRY(cudaMalloc(&ctx->d_cell_of, sizeof(int) * nb));
            CUDA_TRY(cudaMalloc(&ctx->d_order, sizeof(int) * nb));
            ctx->idx_box_cap = nb;
        }
        if ((size_t)n_cells + 1 > ctx->idx_cell_cap) {
            cudaFree(ctx->d_cell_start);
            cudaFree(ctx->d_count);
            cudaFree(ctx->d_cursor);
            cudaFree(ctx->d_cell_lo);
            cudaFree(ctx->d_cell_hi);
            ctx->d_cell_start = ctx->d_count = ctx->d_cursor = nullptr;
            ctx->d_cell_lo = ctx->d_cell_hi = nullptr;
            ctx->idx_cell_cap = 0;
            CUDA_TRY(cudaMalloc(&ctx->d_cell_start, sizeof(int) * (n_cells + 1)));
            CUDA_TRY(cudaMalloc(&ctx->d_count, sizeof(int) * n_cells));
            CUDA_TRY(cudaMalloc(&ctx->d_cursor, sizeof(int) * n_cells));
            CUDA_TRY(cudaMalloc(&ctx->d_cell_lo, sizeof(float4) * n_cells));
            CUDA_TRY(cudaMalloc(&ctx->d_cell_hi, sizeof(float4) * n_cells));
            ctx->idx_cell_cap = (size_t)n_cells + 1;
        }
        if (!ctx->d_overhang)
            CUDA_TRY(cudaMalloc(&ctx->d_overhang, sizeof(unsigned)));
        CUDA_TRY(launch_grid_build(ctx->d_lo, ctx->d_hi, (int)n, ctx->dims, (float)x0, (float)y0, (float)cell, gnx,
                                   gny, ctx->d_cell_of, ctx->d_count, ctx->d_cursor, ctx->d_order,
                                   ctx->d_cell_start, ctx->d_perm, ctx->d_cell_lo, ctx->d_cell_hi,
                                   ctx->d_overhang, ctx->aux));
        CUDA_TRY(cudaStreamSynchronize(ctx->aux));
        unsigned oh_bits = 0;
        CUDA_TRY(cudaMemcpy(&oh_bits, ctx->d_overhang, sizeof(unsigned), cudaMemcpyDeviceToHost));
        float oh;
        std::memcpy(&oh, &oh_bits, 4);
        DevScene &sc = ctx->scene;
        for (int p = 0; p < 6; ++p)
            sc.boxes[p] = ctx->d_perm[p];
        sc.n_boxes = (int)n;
        sc.dims = ctx->dims;
        sc.cell_start = ctx->d_cell_start;
        sc.cell_lo = ctx->d_cell_lo;
        sc.cell_hi = ctx->d_cell_hi;
        sc.gx0 = (float)x0;
        sc.gy0 = (float)y0;
        sc.cell = (float)cell;
        sc.inv_cell = (float)(1.0 / cell);
        sc.gnx = gnx;
        sc.gny = gny;
        sc.overhang = oh;
        ctx->built = true;
        ++ctx->scene_gen;
        return VCM_OK;
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_build: %s", ex.what());
    }
}

vcm_status vcm_compute(vcm_ctx *ctx, const vcm_request *req, float *d_v, uint8_t *d_color, uint32_t *d_bits,
                       vcm_stats *d_stats, void *stream)
{
    float *vv[1] = {d_v};
    uint8_t *cc[1] = {d_color};
    uint32_t *bb[1] = {d_bits};
    return vcm_compute_batch(ctx, req, 1, vv, cc, bb, d_stats, stream);
}

vcm_status vcm_compute_batch(vcm_ctx *ctx, const vcm_request *reqs, uint32_t n, float *const *d_v,
                             uint8_t *const *d_color, uint32_t *const *d_bits, vcm_stats *d_stats, void *stream)
{
    Range range("vcm_compute_batch");
    try {
        vcm_status st = validate_ctx(ctx);
        if (st != VCM_OK)
            return st;
        if (!reqs || n == 0 || !d_v || !d_stats)
            return fail(VCM_E_ARG, "reqs, d_v and d_stats are required and n > 0");
        std::vector<Canon> cs(n);
        for (uint32_t i = 0; i < n; ++i) {
            if ((st = canonicalise(&reqs[i], cs[i])) != VCM_OK)
                return st;
            if (!d_v[i])
                return fail(VCM_E_ARG, "d_v[%u] is NULL", i);
            if ((cs[i].flags & VCM_EMIT_BITS) && (!d_bits || !d_bits[i]))
                return fail(VCM_E_ARG, "VCM_EMIT_BITS needs d_bits[%u]", i);
        }
        std::vector<const Canon *> ptrs;
        std::vector<vcm_tune> shapes;
        for (auto &c : cs) {
            ptrs.push_back(&c);
            shapes.push_back(shape_for(ctx, c));
        }
        std::lock_guard<std::mutex> g(ctx->mu);
        return enqueue_launch(ctx, ctx->direct, ptrs, shapes, d_v, d_color, d_bits, d_stats,
                              static_cast<cudaStream_t>(stream), true);
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_compute_batch: %s", ex.what());
    }
}

vcm_status vcm_submit_batch(vcm_ctx *ctx, const vcm_request *reqs, uint32_t n, uint64_t *tickets)
{
    Range range("vcm_submit_batch");
    try {
        vcm_status st = validate_ctx(ctx);
        if (st != VCM_OK)
            return st;
        if (!reqs || n == 0 || !tickets)
            return fail(VCM_E_ARG, "reqs and tickets are required and n > 0");
        std::vector<std::shared_ptr<Ticket>> grp;
        size_t need = 0;
        for (uint32_t i = 0; i < n; ++i) {
            auto t = std::make_shared<Ticket>();
            if ((st = canonicalise(&reqs[i], t->canon)) != VCM_OK)
                return st;
            need += t->canon.out_bytes() + 1024;
            grp.push_back(t);
        }
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!ctx->built)
            return fail(VCM_E_STATE, "vcm_build has not been called for the current scene");
        if (need + slot_scratch_need(ctx) > ctx->budget)
            return fail(VCM_E_NOMEM, "request needs %zu bytes and a slot's scratch %zu, budget is %zu", need,
                        slot_scratch_need(ctx), ctx->budget);
        const auto now = std::chrono::steady_clock::now();
        for (uint32_t i = 0; i < n; ++i) {
            auto &t = grp[i];
            t->id = ctx->next_ticket++;
            t->shape = shape_for(ctx, t->canon);
            t->t_submit = now;
            ctx->tickets[t->id] = t;
            tickets[i] = t->id;
        }
        ctx->queue.push_back(grp);
        (void)schedule_once(ctx);   // start at once when a slot is free
        ctx->cv.notify_all();
        return VCM_OK;
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_submit_batch: %s", ex.what());
    }
}

vcm_status vcm_submit(vcm_ctx *ctx, const vcm_request *req, uint64_t *ticket)
{
    return vcm_submit_batch(ctx, req, 1, ticket);
}

vcm_status vcm_poll(vcm_ctx *ctx, uint64_t ticket, int32_t wait_ms)
{
    if (!ctx)
        return fail(VCM_E_ARG, "context is NULL");
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end())
        return fail(VCM_E_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    std::shared_ptr<Ticket> t = it->second;
    auto finished = [&] { return t->state == T_DONE || t->state == T_ERROR || t->state == T_CANCELLED; };
    if (wait_ms < 0)
        ctx->cv.wait(lk, finished);
    else if (wait_ms > 0)
        ctx->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), finished);
    switch (t->state) {
    case T_DONE:
        return VCM_OK;
    case T_CANCELLED:
        return fail(VCM_E_CANCELLED, "request %llu was cancelled", (unsigned long long)ticket);
    case T_ERROR:
        return fail(t->err, "%s", t->msg.c_str());
    default:
        return VCM_PENDING;
    }
}

vcm_status vcm_result_get(vcm_ctx *ctx, uint64_t ticket, vcm_result *out)
{
    if (!ctx || !out)
        return fail(VCM_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end())
        return fail(VCM_E_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Ticket &t = *it->second;
    if (t.state != T_DONE)
        return fail(VCM_E_STATE, "request %llu is not finished", (unsigned long long)ticket);
    std::memset(out, 0, sizeof(*out));
    out->v = t.h_v;
    out->color = t.h_color;
    out->bits = t.h_bits;
    out->d_v = t.d_v;
    out->d_color = t.d_color;
    out->d_bits = t.d_bits;
    out->n_viewpoints = (uint64_t)t.canon.n_vp;
    out->words_per_viewpoint = (uint32_t)t.canon.words;
    out->stats = *t.h_stats;
    out->stats.segments = (unsigned long long)t.canon.n_vp * t.canon.P;
    out->latency_ms = std::chrono::duration<double, std::milli>(t.t_done - t.t_submit).count();
    out->queue_ms = std::chrono::duration<double, std::milli>(t.t_launch - t.t_submit).count();
    out->device_ms = t.device_ms;
    out->group_size = t.group_size;
    out->launch_form = t.form;
    out->launch_ms = t.launch_ms;
    out->chain_ms = t.chain_ms;
    return VCM_OK;
}

vcm_status vcm_result_release(vcm_ctx *ctx, uint64_t ticket)
{
    if (!ctx)
        return fail(VCM_E_ARG, "context is NULL");
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->tickets.find(ticket);
        if (it == ctx->tickets.end())
            return fail(VCM_E_ARG, "unknown ticket %llu", (unsigned long long)ticket);
        Ticket &t = *it->second;
        if (t.state == T_QUEUED || t.state == T_RUNNING)
            return fail(VCM_E_STATE, "request %llu is still pending", (unsigned long long)ticket);
        cudaSetDevice(ctx->device);
        release_buffers(ctx, t);
        ctx->tickets.erase(it);
    }
    ctx->cv.notify_all();
    return VCM_OK;
}

vcm_status vcm_cancel(vcm_ctx *ctx, uint64_t ticket)
{
    if (!ctx)
        return fail(VCM_E_ARG, "context is NULL");
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end())
        return fail(VCM_E_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Ticket &t = *it->second;
    if (t.state != T_QUEUED)
        return fail(VCM_E_STATE, "request %llu is already admitted", (unsigned long long)ticket);
    for (auto qit = ctx->queue.begin(); qit != ctx->queue.end(); ++qit) {
        auto &grp = *qit;
        auto pos = std::find_if(grp.begin(), grp.end(), [&](const std::shared_ptr<Ticket> &p) { return p->id == ticket; });
        if (pos != grp.end()) {
            grp.erase(pos);
            if (grp.empty())
                ctx->queue.erase(qit);
            break;
        }
    }
    t.state = T_CANCELLED;
    t.t_done = std::chrono::steady_clock::now();
    ctx->cv.notify_all();
    return VCM_OK;
}

vcm_status vcm_set_slots(vcm_ctx *ctx, uint32_t slots, uint32_t max_batch)
{
    vcm_status st = validate_ctx(ctx);
    if (st != VCM_OK)
        return st;
    if (slots < 1 || slots > 16 || max_batch < 1 || max_batch > 4096)
        return fail(VCM_E_ARG, "slots must be 1..16 and max_batch 1..4096");
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!scheduler_idle(ctx))
            return fail(VCM_E_STATE, "requests are still queued or running");
        ctx->max_batch = max_batch;
    }
    stop_scheduler(ctx);
    for (auto &s : ctx->slots)
        destroy_slot(*s);
    ctx->slots.clear();
    ctx->scratch = 0;
    ctx->last_launched = nullptr;
    return start_scheduler(ctx, slots);
}

vcm_status vcm_get_memory(vcm_ctx *ctx, vcm_memory *out)
{
    if (!ctx || !out)
        return fail(VCM_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(ctx->mu);
    out->budget = ctx->budget;
    out->results = ctx->used;
    out->slot_scratch = ctx->scratch;
    out->slot_scratch_need = slot_scratch_need(ctx);
    out->cached_bits = ctx->cache_bytes;
    out->cache_entries = (uint32_t)ctx->cache.size();
    return VCM_OK;
}

vcm_status vcm_cache_clear(vcm_ctx *ctx)
{
    vcm_status st = validate_ctx(ctx);
    if (st != VCM_OK)
        return st;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        cache_clear(ctx);
    }
    ctx->cv.notify_all();   // freed memory may admit queued requests
    return VCM_OK;
}

vcm_status vcm_set_request_log(vcm_ctx *ctx, const char *path)
{
    vcm_status st = validate_ctx(ctx);
    if (st != VCM_OK)
        return st;
    FILE *f = nullptr;
    if (path) {
        f = std::fopen(path, "a");
        if (!f)
            return fail(VCM_E_ARG, "cannot open %s for appending", path);
    }
    std::lock_guard<std::mutex> g(ctx->log_mu);
    if (ctx->req_log)
        std::fclose(ctx->req_log);
    ctx->req_log = f;
    ctx->log_on.store(f != nullptr, std::memory_order_relaxed);
    return VCM_OK;
}

vcm_status vcm_latency_summary(vcm_ctx *ctx, double *p50_ms, double *p99_ms, uint64_t *completed)
{
    vcm_status st = validate_ctx(ctx);
    if (st != VCM_OK)
        return st;
    if (!p50_ms || !p99_ms || !completed)
        return fail(VCM_E_ARG, "NULL argument");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        lat = ctx->lat_ring;
        *completed = ctx->lat_done;
    }
    *p50_ms = *p99_ms = 0.0;
    if (lat.empty())
        return VCM_OK;
    std::sort(lat.begin(), lat.end());
    // nearest rank: the smallest latency with at least q of the requests at or below it
    auto rank = [&](double q) { return lat[std::max<size_t>(1, (size_t)std::ceil(q * lat.size())) - 1]; };
    *p50_ms = rank(0.50);
    *p99_ms = rank(0.99);
    return VCM_OK;
}

vcm_status vcm_inject(vcm_ctx *ctx, uint32_t kind, uint32_t count)
{
    if (!ctx)
        return fail(VCM_E_ARG, "context is NULL");
    std::lock_guard<std::mutex> g(ctx->mu);
    switch (kind) {
    case VCM_INJECT_NONE:
        if (count != 0)
            return fail(VCM_E_ARG, "VCM_INJECT_NONE takes count 0");
        ctx->inject_spill = ctx->inject_alloc = 0;
        return VCM_OK;
    case VCM_INJECT_SPILL_BUSY:
        ctx->inject_spill = count;
        return VCM_OK;
    case VCM_INJECT_ALLOC_FAIL:
        ctx->inject_alloc = count;
        return VCM_OK;
    default:
        return fail(VCM_E_ARG, "unknown injection kind %u", kind);
    }
}

vcm_status vcm_set_tune(vcm_ctx *ctx, const vcm_tune *tune)
{
    if (!ctx || !tune)
        return fail(VCM_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(ctx->mu);
    if (tune->tile_x == 0) {
        ctx->forced = false;
        return VCM_OK;
    }
    if (tune->tile_x > 256 || tune->tile_y < 1 || tune->tile_y > 256 ||
        tune->tile_x * tune->tile_y > (uint32_t)kMaxTileViewpoints || tune->patch_k > 16 ||
        tune->box_cap < 32 || tune->box_cap > 5000)
        return fail(VCM_E_ARG, "tile sides 1..256 with at most %d viewpoints per tile, patch_k 0..16 (rows per "
                    "pass are capped at 8), box_cap 32..5000", kMaxTileViewpoints);
    ctx->forced = true;
    ctx->forced_tune = *tune;
    return VCM_OK;
}

vcm_status vcm_get_tune(vcm_ctx *ctx, const vcm_request *req, vcm_tune *out)
{
    if (!ctx || !out)
        return fail(VCM_E_ARG, "NULL argument");
    Canon c;
    vcm_status st = canonicalise(req, c);
    if (st != VCM_OK)
        return st;
    std::lock_guard<std::mutex> g(ctx->mu);
    std::vector<vcm_tune> shapes{shape_for(ctx, c)};
    shrink_small_launch(ctx, {&c}, shapes);
    *out = shapes[0];
    DevRequest d{};
    fill_shape(c, *out, d);
    out->patch_k = (uint32_t)d.k_rows;
    return VCM_OK;
}

vcm_status vcm_recolor(vcm_ctx *ctx, const vcm_request *req, const uint32_t *d_bits, float *d_v,
                       uint8_t *d_color, vcm_stats *d_stats, void *stream)
{
    Range range("vcm_recolor");
    try {
        vcm_status st = validate_ctx(ctx);
        if (st != VCM_OK)
            return st;
        if (!d_bits || !d_v || !d_stats)
            return fail(VCM_E_ARG, "d_bits, d_v and d_stats are required");
        Canon c;
        if ((st = canonicalise(req, c)) != VCM_OK)
            return st;
        if (c.flags & VCM_VIEWER)
            return fail(VCM_E_ARG, "vcm_recolor takes target-centric requests only");
        c.flags &= ~(unsigned)VCM_EMIT_BITS;   // the bits are an input here
        if (c.n_vp > (long long)INT32_MAX)
            return fail(VCM_E_ARG, "vcm_recolor takes at most 2^31 - 1 viewpoints");
        const std::vector<const Canon *> cs{&c};
        const std::vector<vcm_tune> shapes{default_tune()};
        const cudaStream_t strm = static_cast<cudaStream_t>(stream);
        std::lock_guard<std::mutex> g(ctx->mu);
        Slot &s = ctx->direct;
        const Layout L = layout_for(cs, shapes);
        if ((st = ensure_slot(ctx, s, L.bytes, 1, 1, strm)) != VCM_OK)
            return st;
        // the previous upload from the pinned descriptors must have completed
        CUDA_TRY(cudaEventSynchronize(s.desc_copied));
        if ((size_t)c.n_vp > ctx->recolor_cap) {
            // earlier work may still read the old list
            CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(ctx->d_recolor_list);
            ctx->d_recolor_list = nullptr;
            ctx->recolor_cap = 0;
            CUDA_TRY(cudaMalloc(&ctx->d_recolor_list, sizeof(int) * (size_t)c.n_vp));
            ctx->recolor_cap = (size_t)c.n_vp;
        }
        if (!ctx->d_recolor_n)
            CUDA_TRY(cudaMalloc(&ctx->d_recolor_n, sizeof(int)));
        float *vv[1] = {d_v};
        uint8_t *cc[1] = {d_color};
        uint32_t *bb[1] = {const_cast<uint32_t *>(d_bits)};   // read only in k_recolor
        fill_desc(s.h_desc, s.d_desc, L, cs, shapes, vv, cc, bb, d_stats, 256, /*blockers=*/false);
        CUDA_TRY(cudaMemcpyAsync(s.d_desc, s.h_desc, L.bytes, cudaMemcpyHostToDevice, strm));
        CUDA_TRY(cudaEventRecord(s.desc_copied, strm));
        CUDA_TRY(cudaMemsetAsync(d_stats, 0, sizeof(vcm_stats), strm));
        const DevRequest *d_reqs = reinterpret_cast<const DevRequest *>(s.d_desc + L.off_reqs);
        const long long *d_vps = reinterpret_cast<const long long *>(s.d_desc + L.off_vps);
        if (ctx->ev_before)
            CUDA_TRY(cudaEventRecord(ctx->ev_before, strm));
        CUDA_TRY(launch_recolor(d_reqs, c.n_vp, ctx->sm_count, ctx->d_recolor_list, ctx->d_recolor_n, strm));
        if (ctx->ev_after)
            CUDA_TRY(cudaEventRecord(ctx->ev_after, strm));
        CUDA_TRY(launch_quantise(d_reqs, d_vps, 1, c.n_vp, strm));
        return VCM_OK;
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_recolor: %s", ex.what());
    }
}

vcm_status vcm_compute_static(const float *lo, const float *hi, uint32_t n_boxes, int32_t dims,
                              const vcm_request *req, float *d_v, uint8_t *d_color, uint32_t *d_bits,
                              vcm_stats *d_stats, void *stream)
{
    Range range("vcm_compute_static");
    try {
        if (dims != 2 && dims != 3)
            return fail(VCM_E_ARG, "dims must be 2 or 3");
        if (n_boxes > VCM_STATIC_MAX_BOXES)
            return fail(VCM_E_ARG, "vcm_compute_static takes at most %u boxes (got %u)", VCM_STATIC_MAX_BOXES,
                        n_boxes);
        if (n_boxes > 0 && (!lo || !hi))
            return fail(VCM_E_ARG, "lo/hi are NULL");
        if (!d_v || !d_stats)
            return fail(VCM_E_ARG, "d_v and d_stats are required");
        {
            // its uploads read host memory that is freed when the call
            // returns, so a captured copy could not be replayed
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            CUDA_TRY(cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap));
            if (cap != cudaStreamCaptureStatusNone)
                return fail(VCM_E_ARG, "vcm_compute_static cannot run on a stream that is being captured");
        }
        Canon c;
        vcm_status st = canonicalise(req, c);
        if (st != VCM_OK)
            return st;
        if (c.dims != dims)
            return fail(VCM_E_ARG, "request dims %d differ from the boxes' dims %d", c.dims, dims);
        if ((c.flags & VCM_EMIT_BITS) && !d_bits)
            return fail(VCM_E_ARG, "VCM_EMIT_BITS needs d_bits");
        if ((unsigned)c.coord_count() > VCM_STATIC_MAX_COORDS)
            return fail(VCM_E_ARG, "vcm_compute_static takes at most %u coordinates (patches_u + patches_w + "
                        "grid_nx + grid_ny + n_layers = %d)", VCM_STATIC_MAX_COORDS, c.coord_count());
        // boxes: lattice checks, world copy n x 3, bounds and largest extent
        const uint32_t n = n_boxes;
        std::vector<float> L((size_t)std::max<uint32_t>(n, 1) * 3, 0.f), H(L.size(), 0.f);
        double x0 = 0, x1 = 1, y0 = 0, y1 = 1, ext = 0;
        if (n) {
            x0 = y0 = 1e30;
            x1 = y1 = -1e30;
        }
        for (uint32_t i = 0; i < n; ++i) {
            for (int k = 0; k < dims; ++k) {
                const float a = lo[(size_t)i * dims + k], b = hi[(size_t)i * dims + k];
                int64_t ua, ub;
                if (!to_units(a, ua) || !to_units(b, ub))
                    return fail(VCM_E_ARG, "box %u coordinate %d is not a finite lattice value within 16384 m", i, k);
                if (ua > ub)
                    return fail(VCM_E_ARG, "box %u has lo > hi on axis %d", i, k);
                L[(size_t)i * 3 + k] = a;
                H[(size_t)i * 3 + k] = b;
            }
            x0 = std::min<double>(x0, L[3 * i]);
            x1 = std::max<double>(x1, H[3 * i]);
            y0 = std::min<double>(y0, L[3 * i + 1]);
            y1 = std::max<double>(y1, H[3 * i + 1]);
            ext = std::max<double>(ext, std::max(H[3 * i] - L[3 * i], H[3 * i + 1] - L[3 * i + 1]));
        }
        const double w = std::max(x1 - x0, 1.0), h = std::max(y1 - y0, 1.0);
        double cell = std::max(std::sqrt(w * h / std::max<uint32_t>(n, 1)) * 1.5, 1.0);
        const double max_cells = 65536.0;
        while ((std::ceil(w / cell) + 1) * (std::ceil(h / cell) + 1) > max_cells)
            cell *= 1.25;
        const int gnx = (int)std::ceil(w / cell) + 1, gny = (int)std::ceil(h / cell) + 1;
        const int n_cells = gnx * gny;

        // place everything in the static scratch array
        CUDA_TRY(init_device());
        void *base = nullptr;
        size_t cap = 0;
        CUDA_TRY(static_scratch(&base, &cap));
        const size_t nb = std::max<uint32_t>(n, 1);
        vcm_tune t = default_tune();
        t.box_cap = (uint32_t)std::max<size_t>(32, nb);   // every candidate list fits: no spill
        std::vector<const Canon *> cs{&c};
        std::vector<vcm_tune> shapes{t};
        const Layout lay = layout_for(cs, shapes);
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t at = off;
            off = align_up(off + bytes, 256);
            return static_cast<char *>(base) + at;
        };
        float *s_lo = reinterpret_cast<float *>(take(nb * 3 * sizeof(float)));
        float *s_hi = reinterpret_cast<float *>(take(nb * 3 * sizeof(float)));
        float4 *s_perm[6];
        for (auto &p : s_perm)
            p = reinterpret_cast<float4 *>(take(nb * 2 * sizeof(float4)));
        int *s_cell_of = reinterpret_cast<int *>(take(nb * sizeof(int)));
        int *s_order = reinterpret_cast<int *>(take(nb * sizeof(int)));
        int *s_count = reinterpret_cast<int *>(take((size_t)n_cells * sizeof(int)));
        int *s_cursor = reinterpret_cast<int *>(take((size_t)n_cells * sizeof(int)));
        int *s_start = reinterpret_cast<int *>(take((size_t)(n_cells + 1) * sizeof(int)));
        float4 *s_cell_lo = reinterpret_cast<float4 *>(take((size_t)n_cells * sizeof(float4)));
        float4 *s_cell_hi = reinterpret_cast<float4 *>(take((size_t)n_cells * sizeof(float4)));
        unsigned *s_overhang = reinterpret_cast<unsigned *>(take(sizeof(unsigned)));
        int *s_work = reinterpret_cast<int *>(take(kWorkHeader * sizeof(int)));   // counters only: no sharing
        int *s_spill = reinterpret_cast<int *>(take(256));   // never written: lists fit box_cap
        char *s_desc = take(lay.bytes);
        if (off > cap)
            return fail(VCM_E_ARG, "request needs %zu bytes of static scratch, the array has %zu", off, cap);

        cudaStream_t sm = static_cast<cudaStream_t>(stream);
        // pageable host sources: each copy has consumed its source when it returns
        CUDA_TRY(cudaMemcpyAsync(s_lo, L.data(), nb * 3 * sizeof(float), cudaMemcpyHostToDevice, sm));
        CUDA_TRY(cudaMemcpyAsync(s_hi, H.data(), nb * 3 * sizeof(float), cudaMemcpyHostToDevice, sm));
        CUDA_TRY(launch_grid_build(s_lo, s_hi, (int)n, dims, (float)x0, (float)y0, (float)cell, gnx, gny, s_cell_of,
                                   s_count, s_cursor, s_order, s_start, s_perm, s_cell_lo, s_cell_hi, s_overhang, sm));
        DevScene sc{};
        for (int p = 0; p < 6; ++p)
            sc.boxes[p] = s_perm[p];
        sc.n_boxes = (int)n;
        sc.dims = dims;
        sc.cell_start = s_start;
        sc.cell_lo = s_cell_lo;
        sc.cell_hi = s_cell_hi;
        sc.gx0 = (float)x0;
        sc.gy0 = (float)y0;
        sc.cell = (float)cell;
        sc.inv_cell = (float)(1.0 / cell);
        sc.gnx = gnx;
        sc.gny = gny;
        // A box is bucketed by its centre, so it reaches at most half its
        // extent past its cell; the host bound avoids reading the device one.
        sc.overhang = (float)(0.5 * ext + 1.0);

        std::vector<char> hdesc(lay.bytes);
        float *vv[1] = {d_v};
        uint8_t *cc[1] = {d_color};
        uint32_t *bb[1] = {d_bits};
        fill_desc(hdesc.data(), s_desc, lay, cs, shapes, vv, cc, bb, d_stats, (int)t.box_cap, /*blockers=*/false);
        CUDA_TRY(cudaMemcpyAsync(s_desc, hdesc.data(), lay.bytes, cudaMemcpyHostToDevice, sm));
        const DevRequest *d_reqs = reinterpret_cast<const DevRequest *>(s_desc + lay.off_reqs);
        const int *d_tiles = reinterpret_cast<const int *>(s_desc + lay.off_tiles);
        const long long *d_vps = reinterpret_cast<const long long *>(s_desc + lay.off_vps);
        int sm_count = 1, dev = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
        const int blocks = std::max(1, std::min(lay.total_tiles, tiles_blocks_per_sm((int)t.box_cap) * sm_count));
        CUDA_TRY(launch_prologue(d_reqs, 1, s_work, (c.flags & VCM_EMIT_BITS) != 0, sm));
        CUDA_TRY(launch_tiles(sc, d_reqs, d_tiles, 1, lay.total_tiles, s_work, s_spill, blocks, (int)t.box_cap,
                              needs_extra(c), c.P >= kTileCheckMinPatches, sm));
        CUDA_TRY(launch_quantise(d_reqs, d_vps, 1, lay.total_vp, sm));
        return VCM_OK;
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_compute_static: %s", ex.what());
    }
}

vcm_status vcm_set_timing_events(vcm_ctx *ctx, void *before_tiles, void *after_tiles)
{
    if (!ctx)
        return fail(VCM_E_ARG, "context is NULL");
    if ((before_tiles == nullptr) != (after_tiles == nullptr))
        return fail(VCM_E_ARG, "give both events or neither");
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->ev_before = static_cast<cudaEvent_t>(before_tiles);
    ctx->ev_after = static_cast<cudaEvent_t>(after_tiles);
    return VCM_OK;
}

vcm_status vcm_autotune(vcm_ctx *ctx, const vcm_request *samples, uint32_t n, vcm_tune *out)
{
    Range range("vcm_autotune");
    try {
        vcm_status st = validate_ctx(ctx);
        if (st != VCM_OK)
            return st;
        if (!samples || n == 0)
            return fail(VCM_E_ARG, "samples are required");
        if (!ctx->built)
            return fail(VCM_E_STATE, "vcm_build has not been called for the current scene");
        std::vector<Canon> cs(n);
        size_t max_vp = 0;
        for (uint32_t i = 0; i < n; ++i) {
            if ((st = canonicalise(&samples[i], cs[i])) != VCM_OK)
                return st;
            cs[i].flags = 0;
            max_vp = std::max<size_t>(max_vp, (size_t)cs[i].n_vp);
        }
        // Shapes are compared at saturation, as a batch runs: a class's
        // samples are replicated in one launch until it holds several waves
        // of tiles, and a shape scores the time per copy of the samples.
        // (Timing a small request alone measures latency on an idle GPU and
        // favours small tiles, which only add per-tile work in a batch.)
        constexpr size_t kMaxCopies = 4096;
        float *d_v = nullptr;
        vcm_stats *d_stats = nullptr;
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CUDA_TRY(cudaMalloc(&d_v, max_vp * sizeof(float)));
        CUDA_TRY(cudaMalloc(&d_stats, kMaxCopies * sizeof(vcm_stats)));
        CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreate(&e0));
        CUDA_TRY(cudaEventCreate(&e1));
        const uint32_t tiles[][2] = {{8, 4}, {8, 8}, {16, 8}, {32, 8}, {16, 16}};
        const uint32_t caps[] = {256, 448, 768};
        // Rows per pass stay automatic: a batch whose classes used different
        // row counts would keep several sweep variants hot at once, a cost
        // that timing one class at a time does not see (the kernel is
        // sensitive to its instruction footprint).
        double best_ms[kTuneClasses];
        vcm_tune best[kTuneClasses];
        bool seen[kTuneClasses] = {false};
        std::lock_guard<std::mutex> g(ctx->mu);
        // Time requests with their shapes, replicated to saturation; the
        // score is the time per copy of the set.
        auto time_set = [&](const std::vector<const Canon *> &mine, const std::vector<vcm_tune> &ts,
                            double &per_copy) -> vcm_status {
            uint32_t cap = 32;
            for (const vcm_tune &t : ts)
                cap = std::max(cap, t.box_cap);
            const long long want = 4LL * tiles_blocks_per_sm((int)cap) * ctx->sm_count;
            std::vector<const Canon *> batch;
            std::vector<vcm_tune> sh;
            long long n_tiles = 0;
            int copies = 0;
            while ((n_tiles < want || copies == 0) && batch.size() + mine.size() <= kMaxCopies) {
                for (size_t i = 0; i < mine.size(); ++i) {
                    batch.push_back(mine[i]);
                    sh.push_back(ts[i]);
                    DevRequest d{};
                    fill_shape(*mine[i], ts[i], d);
                    n_tiles += d.n_tiles;
                }
                ++copies;
            }
            std::vector<float *> vv(batch.size(), d_v);   // the copies share one output (timing only)
            vcm_status st2 = enqueue_launch(ctx, ctx->direct, batch, sh, vv.data(), nullptr, nullptr, d_stats, s,
                                            false, /*adapt=*/false);
            if (st2 != VCM_OK)
                return st2;
            float best_one = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                CUDA_TRY(cudaEventRecord(e0, s));
                if ((st2 = enqueue_launch(ctx, ctx->direct, batch, sh, vv.data(), nullptr, nullptr, d_stats, s, false,
                                          /*adapt=*/false)) != VCM_OK)
                    return st2;
                CUDA_TRY(cudaEventRecord(e1, s));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                best_one = std::min(best_one, ms);
            }
            per_copy = best_one / copies;
            return VCM_OK;
        };
        auto time_shape = [&](const std::vector<const Canon *> &mine, const vcm_tune &t, double &per_copy) {
            return time_set(mine, std::vector<vcm_tune>(mine.size(), t), per_copy);
        };
        for (int cls = 0; cls < kTuneClasses; ++cls) {
            std::vector<const Canon *> mine;
            for (auto &c : cs)
                if (tune_class(c.P) == cls && !(c.flags & VCM_VIEWER))   // viewer shapes are fixed
                    mine.push_back(&c);
            if (mine.empty())
                continue;
            seen[cls] = true;
            // start from the default and move only on a clear (3 %) gain
            best[cls] = default_tune();
            if ((st = time_shape(mine, best[cls], best_ms[cls])) != VCM_OK)
                return st;
            for (auto &tl : tiles)
                for (uint32_t cap : caps) {
                    vcm_tune t{tl[0], tl[1], default_tune().patch_k, cap};
                    double total = 0.0;
                    if ((st = time_shape(mine, t, total)) != VCM_OK)
                        return st;
                    if (total < 0.97 * best_ms[cls]) {
                        best_ms[cls] = total;
                        best[cls] = t;
                    }
                }
        }
        // The classes run together in a batch: keep the tuned shapes only if
        // all samples together, each with its class's shape, beat the
        // default by 3 % as well.
        {
            std::vector<const Canon *> all;
            std::vector<vcm_tune> tuned_sh, default_sh;
            for (auto &c : cs) {
                if (c.flags & VCM_VIEWER)
                    continue;
                all.push_back(&c);
                tuned_sh.push_back(best[tune_class(c.P)]);
                default_sh.push_back(default_tune());
            }
            double t_tuned = 0.0, t_default = 0.0;
            if (!all.empty() && (st = time_set(all, default_sh, t_default)) != VCM_OK)
                return st;
            if (!all.empty() && (st = time_set(all, tuned_sh, t_tuned)) != VCM_OK)
                return st;
            if (!(t_tuned < 0.97 * t_default))
                for (int cls = 0; cls < kTuneClasses; ++cls)
                    best[cls] = default_tune();
        }
        for (int cls = 0; cls < kTuneClasses; ++cls)
            if (seen[cls])
                ctx->tune[cls] = best[cls];
        if (out)
            for (uint32_t i = 0; i < n; ++i)
                out[i] = shape_for(ctx, cs[i]);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        cudaFree(d_v);
        cudaFree(d_stats);
        return VCM_OK;
    } catch (const std::exception &ex) {
        return fail(VCM_E_NOMEM, "vcm_autotune: %s", ex.what());
    }
}

}  // extern "C"
