// vcm_kernels.cu -- sm_103a kernels of the visibility color map engine.
//
//  * grid build: boxes bucketed by footprint centre into a uniform 2D grid
//    (count -> scan -> scatter -> per-cell sort -> permuted copies -> bounds);
//  * tile kernel: persistent blocks draw viewpoint tiles from a queue; each
//    tile culls the scene against the convex hull of (tile, target) using
//    the grid, stages the candidates in shared memory with cp.async, and its
//    warps sweep the tile's viewpoints, lanes over target patch columns and
//    registers over patch rows, deciding each viewpoint->patch segment by a
//    float32 slab test (Def. 2 point-to-point visibility; touching blocks,
//    Def. 4) with an exact float64 re-decision inside a 1e-6 margin band,
//    then summing A cos(theta)/d^2 (or len cos(theta)/d in 2D) per viewpoint;
//  * quantise: colors in L levels from v / v_ref (Def. 1 normalisation).
#include "vcm_internal.h"

#include <cfloat>
#include <climits>
#include <cstdio>
#include <mutex>

namespace vcm {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

// Bounds checks of the checked build (libvcm_checked, compiled with
// VCM_CHECKED): an index outside its buffer sets the request's error word to
// VCM_DEVERR_BOUNDS and the access is skipped; nothing traps.  In the normal
// build the check is the constant true and costs nothing.
#ifdef VCM_CHECKED
__device__ __noinline__ bool in_bounds_slow(long long i, long long n, vcm_stats *st)
{
    if (i >= 0 && i < n)
        return true;
    if (st)
        atomicExch(&st->error, (unsigned)VCM_DEVERR_BOUNDS);
    return false;
}
#define IN_BOUNDS(i, n, st) in_bounds_slow((long long)(i), (long long)(n), (st))
#else
#define IN_BOUNDS(i, n, st) true
#endif

// Box i of a tile's candidate list: staged in shared memory, or (past
// n_smem) through its id in the block's spill region.  The checked build
// replaces an out-of-range id by an empty box, which blocks nothing.
__device__ __forceinline__ void load_box(const float4 *__restrict__ sbox, int n_smem, const int *__restrict__ spill,
                                         const float4 *__restrict__ gbox, int i, int n_boxes, vcm_stats *st,
                                         float4 &lo, float4 &hi)
{
    if (i < n_smem) {
        lo = sbox[2 * i];
        hi = sbox[2 * i + 1];
        return;
    }
    const int s = IN_BOUNDS(i - n_smem, n_boxes, st) ? spill[i - n_smem] : -1;
    if (!IN_BOUNDS(s, n_boxes, st)) {
        lo = make_float4(f_inf(), f_inf(), f_inf(), 0.f);
        hi = make_float4(-f_inf(), -f_inf(), -f_inf(), 0.f);
        return;
    }
    lo = __ldg(&gbox[2 * s]);
    hi = __ldg(&gbox[2 * s + 1]);
}

// Output stores of a request: value of viewpoint vp, occlusion-bit word at
// index `at` (bounds checked in the checked build).
__device__ __forceinline__ void put_v(const DevRequest &R, long long vp, float v)
{
    if (IN_BOUNDS(vp, (long long)R.nx * R.ny * R.nl, R.stats))
        R.v_out[vp] = v;
}
__device__ __forceinline__ void put_word(const DevRequest &R, long long at, uint32_t w)
{
    if (IN_BOUNDS(at, (long long)R.nx * R.ny * R.nl * R.words, R.stats))
        R.bits_out[at] = w;
}

// Hardware reciprocal, at most 1 ulp from 1/d (2^-23 relative); 1/(+0) = +inf.
// The slab-test error bound with it is about 5 u per t value, 10 u per
// margin, still inside the 1e-6 band that is re-decided in float64.
__device__ __forceinline__ float rcp_approx(float d)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}

// ---------------------------------------------------------------------------
// grid build
// ---------------------------------------------------------------------------

__global__ void k_box_cell(const float *__restrict__ lo, const float *__restrict__ hi, int n,
                           float gx0, float gy0, float inv_cell, int gnx, int gny,
                           int *__restrict__ cell_of, int *__restrict__ count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float cx = 0.5f * (lo[3 * i + 0] + hi[3 * i + 0]);
    float cy = 0.5f * (lo[3 * i + 1] + hi[3 * i + 1]);
    int ix = (int)floorf((cx - gx0) * inv_cell);
    int iy = (int)floorf((cy - gy0) * inv_cell);
    ix = min(max(ix, 0), gnx - 1);
    iy = min(max(iy, 0), gny - 1);
    int c = iy * gnx + ix;
    cell_of[i] = c;
    atomicAdd(&count[c], 1);
}

// Exclusive scan of count[0..n) into start[0..n] in three kernels: block
// sums of kScanChunk elements, a one-block scan of the block sums (at most
// 1024 of them: n <= 4M cells), then each block's scan with its offset.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;   // 4096 elements per block

// Exclusive scan of one int per thread over a block of kScanThreads;
// returns the thread's prefix and sets total.
__device__ __forceinline__ int block_exclusive_scan(int x, int &total)
{
    __shared__ int s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, off);
        if (lane >= off)
            incl += t;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        before += w < warp ? s_warp[w] : 0;
        total += s_warp[w];
    }
    __syncthreads();   // s_warp may be reused by the caller's next scan
    return before + incl - x;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *__restrict__ count, int n,
                                                              int *__restrict__ block_sum)
{
    const int base = blockIdx.x * kScanChunk;
    int local = 0;
    for (int i = threadIdx.x; i < kScanChunk && base + i < n; i += kScanThreads)
        local += count[base + i];
    int total;
    (void)block_exclusive_scan(local, total);
    if (threadIdx.x == 0)
        block_sum[blockIdx.x] = total;
}

// One block: exclusive scan of the n_blocks (<= 1024) block sums in place;
// start[n] gets the grand total.
__global__ void __launch_bounds__(1024) k_scan_top(int *__restrict__ block_sum, int n_blocks, int n,
                                                   int *__restrict__ start)
{
    __shared__ int s_part[1024];
    const int t = threadIdx.x;
    const int x = t < n_blocks ? block_sum[t] : 0;
    s_part[t] = x;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? s_part[t - off] : 0;
        __syncthreads();
        s_part[t] += v;
        __syncthreads();
    }
    if (t < n_blocks)
        block_sum[t] = s_part[t] - x;
    if (t == 1023)
        start[n] = s_part[t];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int *__restrict__ count, int n,
                                                            const int *__restrict__ block_off, int *__restrict__ start)
{
    // each thread owns kScanItems consecutive elements of the block's chunk
    const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
    int v[kScanItems], local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? count[base + k] : 0;
        local += v[k];
    }
    int total;
    int run = block_off[blockIdx.x] + block_exclusive_scan(local, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n)
            start[base + k] = run;
        run += v[k];
    }
}

__global__ void k_scatter(const int *__restrict__ cell_of, int n, const int *__restrict__ start,
                          int *__restrict__ cursor, int *__restrict__ order)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int c = cell_of[i];
    int pos = start[c] + atomicAdd(&cursor[c], 1);
    order[pos] = i;
}

// Deterministic order inside each cell: ascending box index (the scatter's
// atomics leave it arbitrary).  Blocks take contiguous ranges of cells, a
// thread each: a cell of at most kSmallCell boxes is sorted in place by its
// thread; larger cells are listed, and the whole block sorts each of them by
// rank (the rank of an id is the number of smaller ids in its cell; ids are
// unique), writing to `tmp` (free after the scatter) and copying back.
constexpr int kSmallCell = 32;

__global__ void __launch_bounds__(kScanThreads) k_sort_cells(const int *__restrict__ start, int n_cells,
                                                             int *__restrict__ order, int *__restrict__ tmp)
{
    __shared__ int s_big[kScanThreads];
    __shared__ int s_n_big;
    for (int c0 = blockIdx.x * kScanThreads; c0 < n_cells; c0 += gridDim.x * kScanThreads) {
        if (threadIdx.x == 0)
            s_n_big = 0;
        __syncthreads();
        const int c = c0 + threadIdx.x;
        if (c < n_cells) {
            const int b = start[c], e = start[c + 1];
            if (e - b > kSmallCell) {
                s_big[atomicAdd(&s_n_big, 1)] = c;
            } else {
                for (int i = b + 1; i < e; ++i) {
                    const int v = order[i];
                    int j = i - 1;
                    while (j >= b && order[j] > v) {
                        order[j + 1] = order[j];
                        --j;
                    }
                    order[j + 1] = v;
                }
            }
        }
        __syncthreads();
        const int n_big = s_n_big;
        for (int k = 0; k < n_big; ++k) {
            const int cb = s_big[k];
            const int b = start[cb], e = start[cb + 1];
            for (int i = b + threadIdx.x; i < e; i += kScanThreads) {
                const int v = order[i];
                int rank = 0;
                for (int j = b; j < e; ++j)
                    rank += order[j] < v;
                tmp[b + rank] = v;
            }
            __syncthreads();
            for (int i = b + threadIdx.x; i < e; i += kScanThreads)
                order[i] = tmp[i];
            __syncthreads();
        }
    }
}

__constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct PermPtrs {
    float4 *p[6];
};

__global__ void k_write_boxes(const float *__restrict__ lo, const float *__restrict__ hi, int n,
                              const int *__restrict__ order, PermPtrs out)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    int id = order[s];
    float L[3] = {lo[3 * id], lo[3 * id + 1], lo[3 * id + 2]};
    float H[3] = {hi[3 * id], hi[3 * id + 1], hi[3 * id + 2]};
    for (int p = 0; p < 6; ++p) {
        const int *a = c_perm[p];
        out.p[p][2 * s] = make_float4(L[a[0]], L[a[1]], L[a[2]], __int_as_float(id));
        out.p[p][2 * s + 1] = make_float4(H[a[0]], H[a[1]], H[a[2]], 0.f);
    }
}

__global__ void k_cell_bounds(const float4 *__restrict__ boxes, const int *__restrict__ start,
                              int gnx, int gny, float gx0, float gy0, float cell,
                              float4 *__restrict__ cell_lo, float4 *__restrict__ cell_hi,
                              unsigned *__restrict__ overhang_bits)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= gnx * gny)
        return;
    float4 lo = make_float4(f_inf(), f_inf(), f_inf(), 0.f);
    float4 hi = make_float4(-f_inf(), -f_inf(), -f_inf(), 0.f);
    int b = start[c], e = start[c + 1];
    for (int s = b; s < e; ++s) {
        float4 l = boxes[2 * s], h = boxes[2 * s + 1];
        lo.x = fminf(lo.x, l.x); lo.y = fminf(lo.y, l.y); lo.z = fminf(lo.z, l.z);
        hi.x = fmaxf(hi.x, h.x); hi.y = fmaxf(hi.y, h.y); hi.z = fmaxf(hi.z, h.z);
    }
    cell_lo[c] = lo;
    cell_hi[c] = hi;
    if (e > b) {
        int ix = c % gnx, iy = c / gnx;
        float x0 = gx0 + ix * cell, y0 = gy0 + iy * cell;
        float oh = fmaxf(fmaxf(x0 - lo.x, hi.x - (x0 + cell)), fmaxf(y0 - lo.y, hi.y - (y0 + cell)));
        oh = fmaxf(oh, 0.f);
        atomicMax(overhang_bits, __float_as_uint(oh));
    }
}

// ---------------------------------------------------------------------------
// tile kernel
// ---------------------------------------------------------------------------

__device__ __forceinline__ float4 world_box_lo(const DevScene &sc, int s) { return __ldg(&sc.boxes[0][2 * s]); }
__device__ __forceinline__ float4 world_box_hi(const DevScene &sc, int s) { return __ldg(&sc.boxes[0][2 * s + 1]); }

struct __align__(16) Plane {
    float x, y, z, c;
};

// n . v, the single evaluation used for hull vertices and box corners alike.
__device__ __forceinline__ float dot3(float nx, float ny, float nz, float x, float y, float z)
{
    return fmaf(nx, x, fmaf(ny, y, nz * z));
}

// True if the box [lo, hi] lies strictly outside one of the hull's planes.
// Each plane's offset was raised by more than twice the worst float32 error
// of dot3 at these coordinate magnitudes, so a box that meets the hull is
// never reported outside.
__device__ __forceinline__ bool outside(const Plane *__restrict__ pl, int np, float4 lo, float4 hi)
{
    for (int i = 0; i < np; ++i) {
        Plane p = pl[i];
        float x = p.x >= 0.f ? lo.x : hi.x;
        float y = p.y >= 0.f ? lo.y : hi.y;
        float z = p.z >= 0.f ? lo.z : hi.z;
        if (dot3(p.x, p.y, p.z, x, y, z) > p.c)
            return true;
    }
    return false;
}

// Exact re-decision of one segment against one box, in float64.  Inputs are
// lattice values (multiples of 2^-10 m, |x| <= 2^14 m): differences are
// exact and every product of two of them needs at most 52 significant bits,
// so the comparisons below are exact.  The running lower bound en/ed and
// upper bound xn/xd of the segment parameter t are kept as fractions with
// positive denominators.
__device__ __noinline__ bool exact_hit(float qu, float qn, float qw, float pu, float pn, float pw,
                                       float4 lo, float4 hi)
{
    const double q[3] = {qu, qn, qw};
    const double p[3] = {pu, pn, pw};
    const double L[3] = {lo.x, lo.y, lo.z};
    const double H[3] = {hi.x, hi.y, hi.z};
    double en = 0.0, ed = 1.0, xn = 1.0, xd = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double d = p[k] - q[k];
        const double a = L[k] - q[k];
        const double b = H[k] - q[k];
        if (d == 0.0) {
            if (a > 0.0 || b < 0.0)
                return false;
            continue;
        }
        double ln, un, den;
        if (d > 0.0) {
            ln = a; un = b; den = d;
        } else {
            ln = -b; un = -a; den = -d;
        }
        if (ln * ed > en * den) {
            en = ln;
            ed = den;
        }
        if (un * xd < xn * den) {
            xn = un;
            xd = den;
        }
    }
    return en * xd <= xn * ed;
}

__constant__ unsigned char c_tri[56][3];

struct TileSmem {
    Plane planes[kMaxPlanes];
    int n_planes;
    int count;
    int item;
    int pad;
    int n_und;
    int helper;   // chunk this block took (-1: a tile from the queue)
    int pub[4];   // record, first chunk, chunks published, offset of the ids in the pool
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Candidate planes of the hull of points P[0..np): for every point triple
// (3D) or pair (2D) whose plane leaves all points on one side, the outward
// normal; of coplanar points only the first triple is kept.  Any normal gives
// a valid half-space once its offset covers every point (below), so float32
// is enough to find them.
__device__ void hull_planes(int dims, const float (*P)[3], int np, TileSmem &sm)
{
    const int t = threadIdx.x;
    float scale = 0.f;
    for (int a = 1; a < np; ++a)
        for (int k = 0; k < 3; ++k)
            scale = fmaxf(scale, fabsf(P[a][k] - P[0][k]));
    scale = fmaxf(scale, 1.f);
    const int n_cand = (dims == 3) ? 56 : 15;
    if (t < n_cand) {
        int i, j, k = -1;
        float n[3];
        if (dims == 3) {
            i = c_tri[t][0]; j = c_tri[t][1]; k = c_tri[t][2];
            float e1[3], e2[3];
            for (int c = 0; c < 3; ++c) {
                e1[c] = P[j][c] - P[i][c];
                e2[c] = P[k][c] - P[i][c];
            }
            n[0] = e1[1] * e2[2] - e1[2] * e2[1];
            n[1] = e1[2] * e2[0] - e1[0] * e2[2];
            n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        } else {
            // pairs (i < j) of 6 points in a fixed order
            int idx = t;
            i = 0;
            while (idx >= np - 1 - i) {
                idx -= np - 1 - i;
                ++i;
            }
            j = i + 1 + idx;
            n[0] = -(P[j][1] - P[i][1]);
            n[1] = P[j][0] - P[i][0];
            n[2] = 0.f;
        }
        const float len = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        const int last = (dims == 3) ? k : j;
        if (len > 1e-6f * scale * scale) {
            const float tol = 1e-5f * len * scale;
            bool pos = false, neg = false, dup = false;
            for (int l = 0; l < np; ++l) {
                const float s = n[0] * (P[l][0] - P[i][0]) + n[1] * (P[l][1] - P[i][1]) +
                                n[2] * (P[l][2] - P[i][2]);
                if (s > tol)
                    pos = true;
                if (s < -tol)
                    neg = true;
                if (fabsf(s) <= tol && l < last && l != i && l != j && l != k)
                    dup = true;
            }
            if (!(pos && neg) && !dup) {
                for (int side = 0; side < 2; ++side) {
                    // side 0: n outward (all points at s <= 0); side 1: -n outward
                    if ((side == 0 && pos) || (side == 1 && neg))
                        continue;
                    const float sg = side ? -1.f : 1.f;
                    const float nx = sg * n[0] / len, ny = sg * n[1] / len, nz = sg * n[2] / len;
                    float c = -f_inf();
                    for (int l = 0; l < np; ++l)
                        c = fmaxf(c, dot3(nx, ny, nz, P[l][0], P[l][1], P[l][2]));
                    c += 0.04f * (fabsf(nx) + fabsf(ny) + fabsf(nz));
                    const int slot = atomicAdd(&sm.n_planes, 1);
                    if (slot < kMaxPlanes)
                        sm.planes[slot] = Plane{nx, ny, nz, c};
                }
            }
        }
    }
    // the six (four in 2D) axis planes of the hull's bounding box
    if (t >= 64 && t < 64 + 2 * dims) {
        const int ax = (t - 64) >> 1;
        const bool upper = ((t - 64) & 1) == 0;
        float m = P[0][ax];
        for (int l = 1; l < np; ++l)
            m = upper ? fmaxf(m, P[l][ax]) : fminf(m, P[l][ax]);
        float n3[3] = {0.f, 0.f, 0.f};
        n3[ax] = upper ? 1.f : -1.f;
        const float c = (upper ? m : -m) + 0.04f;
        const int slot = atomicAdd(&sm.n_planes, 1);
        if (slot < kMaxPlanes)
            sm.planes[slot] = Plane{n3[0], n3[1], n3[2], c};
    }
}

// True if the box [lo, hi] (target frame) certainly (margin > band) blocks
// the segments from q to all four extreme patch centres; see below.
__device__ __forceinline__ bool box_blocks_all(const DevRequest &R, float4 lo, float4 hi, float qu, float qn,
                                               float qw)
{
    const float du0 = R.u_min - qu, du1 = R.u_max - qu;
    const float dn = R.p_n - qn;
    const float dw0 = R.w_min - qw, dw1 = R.w_max - qw;
    const float iu0 = rcp_approx(du0), iu1 = rcp_approx(du1), inn = rcp_approx(dn);
    const float iw0 = rcp_approx(dw0), iw1 = rcp_approx(dw1);
    const float au = lo.x - qu, bu = hi.x - qu, an = lo.y - qn, bn = hi.y - qn;
    const float aw = lo.z - qw, bw = hi.z - qw;
    const float nu0 = (du0 >= 0.f ? au : bu) * iu0, fu0 = (du0 >= 0.f ? bu : au) * iu0;
    const float nu1 = (du1 >= 0.f ? au : bu) * iu1, fu1 = (du1 >= 0.f ? bu : au) * iu1;
    const float nw0 = (dw0 >= 0.f ? aw : bw) * iw0, fw0 = (dw0 >= 0.f ? bw : aw) * iw0;
    const float nw1 = (dw1 >= 0.f ? aw : bw) * iw1, fw1 = (dw1 >= 0.f ? bw : aw) * iw1;
    const float e0 = fmaxf((dn >= 0.f ? an : bn) * inn, 0.f);
    const float x0 = fminf((dn >= 0.f ? bn : an) * inn, 1.f);
    return fminf(fminf(fu0, fw0), x0) - fmaxf(fmaxf(nu0, nw0), e0) > kBand &&
           fminf(fminf(fu1, fw0), x0) - fmaxf(fmaxf(nu1, nw0), e0) > kBand &&
           fminf(fminf(fu0, fw1), x0) - fmaxf(fmaxf(nu0, nw1), e0) > kBand &&
           fminf(fminf(fu1, fw1), x0) - fmaxf(fmaxf(nu1, nw1), e0) > kBand;
}

// True if the box certainly blocks the segments from all four corner
// viewpoints (x0|x1, y0|y1, layer z) of a tile to the four extreme patch
// centres (see the whole-tile check in the tile kernel).  Not inlined: it
// runs once per tile and would add to the tile kernel's registers.
__device__ __noinline__ bool box_blocks_tile(const DevRequest &R, float4 lo, float4 hi, float x0, float x1, float y0,
                                             float y1, float z)
{
    for (int c = 0; c < 4; ++c) {
        const float qx = (c & 1) ? x1 : x0, qy = (c & 2) ? y1 : y0;
        const float qu = R.au == 0 ? qx : (R.au == 1 ? qy : z);
        const float qn = R.an == 0 ? qx : (R.an == 1 ? qy : z);
        const float qw = R.dims == 3 ? (R.aw == 0 ? qx : (R.aw == 1 ? qy : z)) : 0.f;
        if (!box_blocks_all(R, lo, hi, qu, qn, qw))
            return false;
    }
    return true;
}

// True if one of the first `nb` (<= 32) staged boxes certainly blocks the
// segments from q to all four extreme patch centres.  On the target plane the
// points whose segment to q meets a convex box form a convex set (a segment
// from q to any point between two blocked ones crosses the box between their
// two hit points), and every patch centre lies in the rectangle spanned by
// the extreme ones, so such a box blocks every patch.  Lanes take one box
// each; only float32 margins above the band count, so the answer is exact.
__device__ __forceinline__ bool one_box_blocks_all(const DevRequest &R, const float4 *__restrict__ sbox, int nb,
                                                   float qu, float qn, float qw)
{
    const int lane = threadIdx.x & 31;
    const float du0 = R.u_min - qu, du1 = R.u_max - qu;
    const float dn = R.p_n - qn;
    const float dw0 = R.w_min - qw, dw1 = R.w_max - qw;
    bool full = false;
    if (lane < nb) {
        const float iu0 = rcp_approx(du0), iu1 = rcp_approx(du1), inn = rcp_approx(dn);
        const float iw0 = rcp_approx(dw0), iw1 = rcp_approx(dw1);
        const float4 lo = sbox[2 * lane], hi = sbox[2 * lane + 1];
        const float au = lo.x - qu, bu = hi.x - qu, an = lo.y - qn, bn = hi.y - qn;
        const float aw = lo.z - qw, bw = hi.z - qw;
        const float nu0 = (du0 >= 0.f ? au : bu) * iu0, fu0 = (du0 >= 0.f ? bu : au) * iu0;
        const float nu1 = (du1 >= 0.f ? au : bu) * iu1, fu1 = (du1 >= 0.f ? bu : au) * iu1;
        const float nw0 = (dw0 >= 0.f ? aw : bw) * iw0, fw0 = (dw0 >= 0.f ? bw : aw) * iw0;
        const float nw1 = (dw1 >= 0.f ? aw : bw) * iw1, fw1 = (dw1 >= 0.f ? bw : aw) * iw1;
        const float e0 = fmaxf((dn >= 0.f ? an : bn) * inn, 0.f);
        const float x0 = fminf((dn >= 0.f ? bn : an) * inn, 1.f);
        const bool c00 = fminf(fminf(fu0, fw0), x0) - fmaxf(fmaxf(nu0, nw0), e0) > kBand;
        const bool c10 = fminf(fminf(fu1, fw0), x0) - fmaxf(fmaxf(nu1, nw0), e0) > kBand;
        const bool c01 = fminf(fminf(fu0, fw1), x0) - fmaxf(fmaxf(nu0, nw1), e0) > kBand;
        const bool c11 = fminf(fminf(fu1, fw1), x0) - fmaxf(fmaxf(nu1, nw1), e0) > kBand;
        full = c00 && c10 && c01 && c11;
    }
    return __any_sync(kFull, full);
}

// Planes of the pyramid with apex q and base the rectangle [u_lo, u_hi] x
// [w_lo, w_hi] of patch centres (2D: the triangle q, segment ends), in the
// target frame (u, n, w).  Every segment from q to a patch centre in the
// rectangle lies in it, so a box outside one of the planes meets none of
// them.  Each plane's offset is the largest float32
// evaluation over all the pyramid's points plus the same margin as the tile
// hull, so the half-space holds the whole pyramid whatever the plane's
// orientation; a degenerate plane only culls less.  Lanes 0..5 each write
// one plane (NaN-free: degenerate normals are dropped); returns the count.
// Not inlined: each sweep variant would carry a copy (1 % on the 3D step).
__device__ __noinline__ int pyramid_planes(const DevRequest &R, float qu, float qn, float qw, float u_lo, float u_hi,
                                           float w_lo, float w_hi, Plane *out)
{
    const int lane = threadIdx.x & 31;
    // rectangle corners in order (u_min,w_min) (u_max,w_min) (u_max,w_max) (u_min,w_max)
    const float P[5][3] = {{qu, qn, qw},
                           {u_lo, R.p_n, w_lo},
                           {u_hi, R.p_n, w_lo},
                           {u_hi, R.p_n, w_hi},
                           {u_lo, R.p_n, w_hi}};
    float nx = 0.f, ny = 0.f, nz = 0.f;
    bool ok = false;
    if (lane == 0) {
        // the target plane: segments stay on q's side of it
        ny = (R.p_n > qn) ? 1.f : -1.f;
        ok = R.p_n != qn;
    } else if (lane <= 4) {
        const int e = lane - 1, f = lane & 3;   // rectangle edge e -> f
        const float eu = (e == 0 || e == 3) ? u_lo : u_hi, ew = (e < 2) ? w_lo : w_hi;
        const float fu = (f == 0 || f == 3) ? u_lo : u_hi, fw = (f < 2) ? w_lo : w_hi;
        if (R.dims == 3) {
            const float ax = eu - qu, ay = R.p_n - qn, az = ew - qw;
            const float bx = fu - qu, by = R.p_n - qn, bz = fw - qw;
            nx = ay * bz - az * by;
            ny = az * bx - ax * bz;
            nz = ax * by - ay * bx;
        } else if (e < 2) {
            // 2D: lines from q through the two segment ends, normal in the (u, n) plane
            nx = -(R.p_n - qn);
            ny = eu - qu;
        }
        const float len = sqrtf(nx * nx + ny * ny + nz * nz);
        ok = len > 0.f;
        if (ok) {
            nx /= len; ny /= len; nz /= len;
            // outward: away from a point inside the pyramid
            const float cu = 0.5f * (qu + 0.5f * (u_lo + u_hi)), cn = 0.5f * (qn + R.p_n);
            const float cw = 0.5f * (qw + 0.5f * (w_lo + w_hi));
            if (dot3(nx, ny, nz, cu, cn, cw) > dot3(nx, ny, nz, qu, qn, qw)) {
                nx = -nx; ny = -ny; nz = -nz;
            }
        }
    }
    float c = -f_inf();
    if (ok) {
        for (int l = 0; l < 5; ++l)
            c = fmaxf(c, dot3(nx, ny, nz, P[l][0], P[l][1], P[l][2]));
        c += 0.04f * (fabsf(nx) + fabsf(ny) + fabsf(nz));
    }
    const unsigned okm = __ballot_sync(kFull, ok && lane <= 4);
    if (ok && lane <= 4)
        out[__popc(okm & ((1u << lane) - 1u))] = Plane{nx, ny, nz, c};
    __syncwarp();
    return __popc(okm);
}

// One viewpoint swept by one warp.  Lane l owns patch column
// cp * nuc + (l % nuc) and rows (rp * K + m) * groups + l / nuc, m < K.
// The t-interval of a segment along u depends only on its column, along n
// only on the viewpoint and along w only on its row, so the u and n parts
// of the slab test are formed once per box and column, and each row adds
// its w interval.
// Does a viewpoint at normal coordinate qn see the measured side of the
// target?  One-sided: n.(q - p) > 0.  Two-sided: anywhere off its plane.
__device__ __forceinline__ bool facing(const DevRequest &R, float qn)
{
    return (R.flags & VCM_TWO_SIDED) ? qn != R.p_n : R.sn * (qn - R.p_n) > 0.f;
}

// Field-of-view cone (Section III-B, Table II): is q inside the cone of the
// patch at q - r, a.r >= c |r|?  r comes in target-frame components
// (u, n, w), each the rounded float difference q - p; the test runs in world
// order x, y, z with one float32 rounding per operation (no fused
// multiply-add), as the request header states, which errs in the margin by
// at most about 10.5 u |r|: only pairs within 1e-6 |r| of the cone's edge
// can be decided differently from the exact inequality.
__device__ __forceinline__ bool in_cone_inline(const DevRequest &R, float ru, float rn, float rw)
{
    const float r0 = R.au == 0 ? ru : (R.an == 0 ? rn : rw);
    const float r1 = R.au == 1 ? ru : (R.an == 1 ? rn : rw);
    const float r2 = R.au == 2 ? ru : (R.an == 2 ? rn : rw);
    float d = __fadd_rn(__fmul_rn(R.cone_a[0], r0), __fmul_rn(R.cone_a[1], r1));
    d = __fadd_rn(d, __fmul_rn(R.cone_a[2], r2));
    if (R.flags & VCM_TWO_SIDED)
        d = fabsf(d);
    float rr = __fadd_rn(__fmul_rn(r0, r0), __fmul_rn(r1, r1));
    rr = __fadd_rn(rr, __fmul_rn(r2, r2));
    return d >= __fmul_rn(R.cone_c, __fsqrt_rn(rr));
}

// The same, not inlined, for the tile kernel's sweep (keeps its code small).
__device__ __noinline__ bool in_cone(const DevRequest &R, float ru, float rn, float rw)
{
    return in_cone_inline(R, ru, rn, rw);
}

// One variant for either sign of the row offsets w - q_w (a per-row sign
// mask): a viewpoint layer inside the target's height range and one outside
// it then run the same code, which halves the sweep's hot instruction
// footprint (a split by sign made the 3D workload 10 % slower).
template <int K, bool EXTRA>
__device__ __forceinline__ float sweep_viewpoint(const DevRequest &R, const float4 *__restrict__ sbox,
                                                 int n_smem, const int *__restrict__ spill, int count,
                                                 const float4 *__restrict__ gbox, float qu, float qn,
                                                 float qw, bool front, long long vp, Plane *pyr,
                                                 bool use_pyr, unsigned long long &tests, unsigned &rechecks,
                                                 int n_boxes)
{
    const int lane = threadIdx.x & 31;
    const int nuc = R.nuc, G = R.groups;
    const int c_in = lane % nuc, g = lane / nuc;
    const bool lane_ok = g < G;
    const float dn = R.p_n - qn;
    const float inv_n = rcp_approx(dn);
    const bool sgn_n = dn >= 0.f;
    const bool want_bits = (R.flags & VCM_EMIT_BITS) && R.bits_out;
    const bool is3d = R.dims == 3;
    // strict: any blocked patch zeroes the viewpoint, so the first one ends it
    const bool strict = (R.flags & VCM_STRICT) != 0;
    const bool strict_exit = strict && !want_bits;
    bool strict_fail = false;
    const float *__restrict__ w_coord = R.w_coord;
    float sum = 0.f, comp = 0.f;

    for (int cp = 0; cp < R.col_passes && !(strict_exit && strict_fail); ++cp) {
        const int iu = cp * nuc + c_in;
        const bool col_ok = lane_ok && iu < R.nu;
        const float pu = R.u_coord[col_ok ? iu : 0];
        const float du = pu - qu;
        const float inv_u = rcp_approx(du);
        const bool sgn_u = du >= 0.f;
        const float ru = qu - pu, rn = qn - R.p_n;
        const float col_d2 = fmaf(ru, ru, rn * rn);
        // measure x |r| cos(theta); a two-sided target is measured from either side
        const float m_s = R.measure * ((EXTRA && (R.flags & VCM_TWO_SIDED)) ? fabsf(rn) : R.sn * rn);
        // The measure: a plain sum over each group of up to 8 of the lane's
        // rows (error <= 7u of the group's total, the terms being >= 0), and a
        // Neumaier-compensated sum of the group totals, so the bound holds for
        // any patch count.
        float psum = 0.f;
        auto add_group = [&](float &g) {
            const float tsum = sum + g;
            if (fabsf(sum) >= fabsf(g))
                comp += (sum - tsum) + g;
            else
                comp += (g - tsum) + sum;
            sum = tsum;
            g = 0.f;
        };
        for (int rp = 0; rp < R.row_passes && !(strict_exit && strict_fail); ++rp) {
            // per row: its w offset dw and the band of its test in w units,
            // tau |dw|; -inf once the row is blocked (or past the patch grid)
            float dwv[K], thr[K];
            unsigned valid = 0, sgnw = 0;
#pragma unroll
            for (int m = 0; m < K; ++m) {
                const int iw = (rp * K + m) * G + g;
                const bool ok = col_ok && iw < R.nw;
                const float dw = w_coord[ok ? iw : 0] - qw;
                dwv[m] = dw;
                if (dw >= 0.f)
                    sgnw |= 1u << m;
                thr[m] = ok ? kBand * fabsf(dw) : -f_inf();
                if (ok)
                    valid |= 1u << m;
            }
            unsigned alive = valid;
            if (!__any_sync(kFull, alive != 0))
                continue;
            // The pyramid filter for this pass: apex q, base the rectangle
            // of the patch centres the pass covers (its columns by its rows),
            // so a box whose shadow misses them is dropped before its rows
            // are tested.
            int npyr = 0;
            if (use_pyr) {
                const int c0 = cp * nuc, c1 = min(R.nu, c0 + nuc) - 1;
                const int r0 = rp * K * G, r1 = min(R.nw, r0 + K * G) - 1;
                const float ua = R.u_coord[c0], ub = R.u_coord[c1], wa = w_coord[r0], wb = w_coord[r1];
                __syncwarp();   // the previous pass has done with the planes
                npyr = pyramid_planes(R, qu, qn, qw, fminf(ua, ub), fmaxf(ua, ub), fminf(wa, wb), fmaxf(wa, wb), pyr);
            }
            int nb = 0;
            bool done = false;
            for (int base = 0; base < count && !done; base += 32) {
              // lanes over boxes: which of the next 32 candidates meet the
              // viewpoint's pyramid at all
              unsigned todo;
              {
                const int i = base + lane;
                bool cand = false;
                if (i < count && npyr == 0) {
                    cand = true;
                } else if (i < count) {
                    float4 lo, hi;
                    load_box(sbox, n_smem, spill, gbox, i, n_boxes, R.stats, lo, hi);
                    cand = !outside(pyr, npyr, lo, hi);
                }
                todo = __ballot_sync(kFull, cand);
              }
              while (todo) {
                const int i = base + __ffs(todo) - 1;
                todo &= todo - 1;
                float4 lo, hi;
                load_box(sbox, n_smem, spill, gbox, i, n_boxes, R.stats, lo, hi);
                const float a_u = lo.x - qu, b_u = hi.x - qu;
                const float a_n = lo.y - qn, b_n = hi.y - qn;
                const float tnu = (sgn_u ? a_u : b_u) * inv_u;
                const float tfu = (sgn_u ? b_u : a_u) * inv_u;
                const float tnn = (sgn_n ? a_n : b_n) * inv_n;
                const float tfn = (sgn_n ? b_n : a_n) * inv_n;
                const float pre_e = fmaxf(fmaxf(tnu, tnn), 0.f);
                const float pre_x = fminf(fminf(tfu, tfn), 1.f);
                // no row of this column can meet the box: skip the rows
                if (__all_sync(kFull, alive == 0 || (pre_x - pre_e) < -kBand))
                    continue;
                ++nb;   // boxes whose rows are tested
                // The column's segment is inside the box's u and n slabs for
                // t in [pre_e, pre_x]; a row meets the box when the w offsets
                // the segment takes there, t * dw, reach the box's w extent
                // [a_w, b_w]: e1 = a_w - (the larger end) < 0 and e2 = (the
                // smaller end) - b_w < 0.  Both are t-margins times |dw|, so the
                // band is tau |dw|, and the column's own margin pre_x - pre_e
                // joins them (a hit needs it above tau; below -tau no row
                // meets the box).  The w extent of a 2D request is unbounded.
                const float lm = pre_x - pre_e;
                const bool lane_sure = lm > kBand;
                float a_w = lo.z - qw, b_w = hi.z - qw;
                if (R.dims != 3) {
                    a_w = -f_inf();
                    b_w = f_inf();
                }
                if (lm < -kBand) {   // e1 and e2 are +inf or NaN: no row enters
                    a_w = f_inf();
                    b_w = -f_inf();
                }
#pragma unroll
                for (int m = 0; m < K; ++m) {
                    const bool sp = (sgnw >> m) & 1u;
                    const float e1 = fmaf(-(sp ? pre_x : pre_e), dwv[m], a_w);
                    const float e2 = fmaf(sp ? pre_e : pre_x, dwv[m], -b_w);
                    const float mm = fmaxf(e1, e2);
                    if (mm <= thr[m] && ((alive >> m) & 1u)) {
                        bool hit = lane_sure && mm < -thr[m];
                        if (!hit) {
                            const int iw = (rp * K + m) * G + g;
                            hit = exact_hit(qu, qn, qw, pu, R.p_n, w_coord[iw], lo, hi);
                            ++rechecks;
                        }
                        if (hit) {
                            thr[m] = -f_inf();
                            alive &= ~(1u << m);
                        }
                    }
                }
                if (__all_sync(kFull, alive == 0) || (strict_exit && __any_sync(kFull, alive != valid))) {
                    done = true;
                    break;
                }
              }
            }
            tests += (unsigned long long)nb * K;
            if (strict)
                strict_fail |= __any_sync(kFull, alive != valid);
            // the blocked bits, and the visible measure of the unblocked rows
            if (want_bits) {
#pragma unroll
                for (int m = 0; m < K; ++m) {
                    if (((valid & ~alive) >> m) & 1u) {
                        const int iw = (rp * K + m) * G + g;
                        const int j = iw * R.nu + iu;
                        if (IN_BOUNDS(vp * R.words + (j >> 5), (long long)R.nx * R.ny * R.nl * R.words, R.stats))
                            atomicOr(&R.bits_out[vp * R.words + (j >> 5)], 1u << (j & 31));
                    }
                }
            }
            const unsigned open = front && !strict_fail ? (valid & alive) : 0u;
            if (__any_sync(kFull, open != 0u)) {
#pragma unroll
                for (int m = 0; m < K; ++m) {
                    if (!((open >> m) & 1u))
                        continue;
                    // |r|^2 = (ru^2 + rn^2) of the column + rw^2 of the row;
                    // rw = q_w - w is the row's offset negated (round to
                    // nearest is symmetric, so exactly -dw)
                    const float rw = -dwv[m];
                    if (EXTRA && R.cone && !in_cone(R, ru, rn, rw))
                        continue;   // q is outside this patch's field of view
                    const float d2 = fmaf(rw, rw, col_d2);
                    float term;
                    if (is3d) {
                        const float ir = rsqrtf(d2);
                        term = m_s * (ir * ir * ir);   // A |r| cos(theta) / |r|^3
                    } else {
                        term = m_s / d2;               // len |r| cos(theta) / |r|^2
                    }
                    // an add the compiler cannot fuse with the term's
                    // product, so every specialised copy of this loop
                    // rounds the same way
                    psum = __fadd_rn(psum, term);
                }
            }
            // a group closes after every 8 of the lane's rows (K divides 8, so
            // the grouping and the result do not depend on K) and at the end
            // of the column pass
            if (((rp + 1) * K) % 8 == 0 || rp + 1 == R.row_passes)
                add_group(psum);
        }
        add_group(psum);   // what a strict early exit left
    }
    float v = sum + comp;
    // fixed-order butterfly: every lane ends with the same value
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(kFull, v, off);
    return strict_fail ? 0.f : v;
}

// Viewer-centric cell (VCM_VIEWER): one segment from the cell q to the
// viewer p (world frame) against the candidate boxes, nearest first; the
// cell's value is the visual angle (2D, Eq. 1) or solid angle (3D) of an
// object of size S at distance D facing the viewer, 0 when blocked or D = 0.
__device__ __forceinline__ float viewer_cell(const DevRequest &R, const float4 *__restrict__ sbox, int n_smem,
                                             const int *__restrict__ spill, int count,
                                             const float4 *__restrict__ gbox, float qx, float qy, float qz,
                                             bool &blocked, unsigned long long &tests, unsigned &rechecks,
                                             int n_boxes)
{
    const float px = R.u_min, py = R.p_n, pz = R.w_min;
    const float dx = px - qx, dy = py - qy, dz = pz - qz;
    const float ix = rcp_approx(dx), iy = rcp_approx(dy), iz = rcp_approx(dz);
    blocked = false;
    for (int i = 0; i < count && !blocked; ++i) {
        float4 lo, hi;
        load_box(sbox, n_smem, spill, gbox, i, n_boxes, R.stats, lo, hi);
        ++tests;
        const float ax = lo.x - qx, bx = hi.x - qx, ay = lo.y - qy, by = hi.y - qy, az = lo.z - qz, bz = hi.z - qz;
        const float enter = fmaxf(fmaxf((dx >= 0.f ? ax : bx) * ix, (dy >= 0.f ? ay : by) * iy),
                                  fmaxf((dz >= 0.f ? az : bz) * iz, 0.f));
        const float exit_ = fminf(fminf((dx >= 0.f ? bx : ax) * ix, (dy >= 0.f ? by : ay) * iy),
                                  fminf((dz >= 0.f ? bz : az) * iz, 1.f));
        const float mv = exit_ - enter;
        if (mv >= -kBand) {
            blocked = mv > kBand;
            if (!blocked) {
                ++rechecks;
                blocked = exact_hit(qx, qy, qz, px, py, pz, lo, hi);
            }
        }
    }
    const float D = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    if (blocked || !(D > 0.f))
        return 0.f;
    const float S = R.measure;
    if (R.dims == 2)
        return 2.f * atanf(S / (2.f * D));
    return 4.f * asinf(S * S / fmaf(4.f * D, D, S * S));
}


// Cull one box against the hull planes and, if it may matter, add it to the
// tile's candidate list (shared memory, then the block's spill region).
__device__ __forceinline__ void add_candidate(const float4 *__restrict__ world, const Plane *planes, int n_planes,
                                              int s, TileSmem &sm, int *s_ids, int box_cap, int *spill,
                                              int spill_slot, const DevRequest &R, int n_boxes)
{
    if (outside(planes, n_planes, world[2 * s], world[2 * s + 1]))
        return;
    const int pos = atomicAdd(&sm.count, 1);
    if (pos < box_cap)
        s_ids[pos] = s;
    else if (spill_slot >= 0) {
        if (IN_BOUNDS(pos - box_cap, n_boxes, R.stats))
            spill[pos - box_cap] = s;
    } else {
        R.stats->error = VCM_DEVERR_SPILL_WAIT;   // no spill region: the result is flagged
    }
}

// EXTRA: the instantiation for launches that hold a two-sided or cone
// request; the common one carries none of that code (the tile kernel is
// sensitive to its instruction footprint).
// Five blocks per SM: the compiler then fits the kernel in 94 registers
// without spilling, and the fifth block hides more of the dependency and
// barrier latency that bound it (4 -> 5 blocks: 3D step -5 %, a 256-request
// batch -11 %; 6 blocks spill and lose on large scenes).
// TILE_CHECK: the instantiation with the whole-tile check below, for
// launches whose requests all have many patches (the host picks it).  It
// decides whole tiles, which pays when a viewpoint's own work is large (the
// 100,000-box scene with 64 x 32 patches: -10 %); in the other instantiation
// its code alone cost a few % on smaller requests.
//
// CHUNKS: the second pass's instantiation, which takes the published chunks
// and holds none of the tile pass's code (the cull, the sort, the checks and
// the publication), so its registers and instructions fit the sweep alone.
//
// Occupancy: the tile pass runs 6 blocks per SM (80 registers) and the chunk
// pass 7 (72 registers).  Both spill some registers at these bounds, and
// still the extra warps hide more latency than the spills cost.  Against 5
// blocks for both (96 registers, no spills in the common instantiations):
// 100,000-box step 4.23 -> 3.86 ms, 5,000-box step 0.354 -> 0.333 ms,
// 256-request batch 91.5 -> 87.9 ms; 7 blocks for the tile pass too made
// the batch 15 % slower.
template <bool EXTRA, bool TILE_CHECK, bool CHUNKS>
__global__ void __launch_bounds__(kThreads, CHUNKS ? 7 : 6)
k_tiles(DevScene sc, const DevRequest *__restrict__ reqs, const int *__restrict__ tile_prefix,
        int n_req, int total_tiles, int *__restrict__ work, int *__restrict__ spill_all, int box_cap,
        int one_tile, int *__restrict__ spill_busy, int spill_slots, int share, int claim_rounds)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *s_box = reinterpret_cast<float4 *>(smem_raw);
    int *s_ids = reinterpret_cast<int *>(smem_raw + (size_t)box_cap * 32);
    __shared__ TileSmem sm;
    __shared__ float s_pts[8][3];
    __shared__ DevRequest s_req;
    __shared__ int s_next;
    __shared__ Plane s_pyr[kWarps][6];
    __shared__ int s_req_idx;
    __shared__ int s_next2;                     // cursor of the undecided list
    __shared__ int s_und[kMaxTileViewpoints];   // viewpoints left by the one-box check
    __shared__ int s_rowpre[kThreads], s_rowx[kThreads], s_wsum[kWarps];   // cell-row spans
    __shared__ int s_passb[kPassCap], s_passn[kPassCap], s_passp[kPassCap + 1], s_wsum2[kWarps], s_npass;
    __shared__ int s_hist[kDistClasses];   // counting sort of long candidate lists

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int s_spill_slot;
    if (tid == 0) {
        s_req_idx = -1;
        s_npass = 0;
        sm.item = -1;
        // A persistent block owns spill region blockIdx.x.  A one-tile block
        // claims a free region for the length of its tile.  There are as
        // many regions as blocks fit on the GPU, so a probe normally succeeds
        // at once; if every region is held (blocks of a preempted launch keep
        // theirs), it probes again after a pause, at most claim_rounds times
        // (kClaimRounds by default: a few ms), and then runs without one and
        // flags the result.
        int slot = (int)blockIdx.x;
        if (one_tile) {
            slot = -1;
            const int start = (int)(blockIdx.x % (unsigned)spill_slots);
            for (int round = 0; round < claim_rounds && slot < 0; ++round) {
                for (int probe = 0; probe < spill_slots && slot < 0; ++probe) {
                    const int c = (start + probe) % spill_slots;
                    if (atomicCAS(&spill_busy[c], 0, 1) == 0)
                        slot = c;
                }
                if (slot < 0)
                    __nanosleep(2000);
            }
        }
        s_spill_slot = slot;
    }
    __syncthreads();
    const int spill_slot = s_spill_slot;
    // the chunk pass reads no spill region (and has more blocks than regions)
    int *spill = CHUNKS ? nullptr : spill_all + (size_t)max(spill_slot, 0) * sc.n_boxes;

    for (;;) {
        // thread 0 takes the next tile, copies its request and lays out the
        // hull points (one barrier for all of it).  With one_tile, block b
        // does tile b only and exits, so blocks of concurrent launches
        // interleave (a persistent grid would hold every SM to the end).
        // The second pass (CHUNKS, share == 2) takes the chunks the first published,
        // in order, and no tiles.
        if (tid == 0) {
            int took = -1, it;
            if (CHUNKS) {
                const int h = atomicAdd(work + 3, 1);
                took = h < min(__ldcg(work + 2), kChunkCap) ? h : -1;
            }
            if (took >= 0) {
                const int rec = __ldcg(work + kWorkHeader + kChunkOff + (size_t)(2 + kChunkVp) * took);
                it = __ldcg(work + kWorkHeader + kRecOff + (size_t)kRecInts * rec);
            } else if (CHUNKS) {
                it = total_tiles;
            } else {
                it = one_tile ? (sm.item == -2 ? total_tiles : (int)blockIdx.x) : atomicAdd(work, 1);
                // Queue order: last tile first, and within a request the
                // layers interleaved (consecutive items are one tile position
                // in every layer).  Measured on the 3D workload with the
                // target facing each of +-x and +-y: 3-14 % faster than the
                // plain order, never slower; either change alone was not.
                it = it < total_tiles ? total_tiles - 1 - it : total_tiles;
            }
            sm.item = it;
            sm.helper = took;
            if (it < total_tiles) {
                // request of this tile: last r with tile_prefix[r] <= it
                int lo_r = 0, hi_r = n_req - 1;
                while (lo_r < hi_r) {
                    const int mid = (lo_r + hi_r + 1) >> 1;
                    if (tile_prefix[mid] <= it)
                        lo_r = mid;
                    else
                        hi_r = mid - 1;
                }
                if (lo_r != s_req_idx) {   // consecutive tiles mostly share a request
                    s_req = reqs[lo_r];
                    s_req_idx = lo_r;
                }
                {
                    // tile index within its request, layers interleaved
                    const int t0 = it - tile_prefix[lo_r];
                    const int nl = s_req.nl, pl = s_req.tiles_x * s_req.tiles_y;
                    sm.pad = (t0 % nl) * pl + t0 / nl;
                }
                const DevRequest &Q = s_req;
                const int t0 = sm.pad, pl = Q.tiles_x * Q.tiles_y;
                const int ly = t0 / pl, t1 = t0 - ly * pl;
                const int ty0 = t1 / Q.tiles_x, tx0 = t1 - ty0 * Q.tiles_x;
                const int x0 = tx0 * Q.tile_x, x1 = min(Q.nx, x0 + Q.tile_x) - 1;
                const int y0 = ty0 * Q.tile_y, y1 = min(Q.ny, y0 + Q.tile_y) - 1;
                const float z = Q.z_coord[ly];
                sm.n_planes = 0;
                sm.count = 0;
                sm.n_und = 0;
                s_next = 0;
                s_next2 = 0;
                const float X[2] = {Q.x_coord[x0], Q.x_coord[x1]};
                const float Y[2] = {Q.y_coord[y0], Q.y_coord[y1]};
                for (int c = 0; c < 4; ++c) {
                    s_pts[c][0] = X[c & 1];
                    s_pts[c][1] = Y[c >> 1];
                    s_pts[c][2] = (Q.dims == 3) ? z : 0.f;
                }
                if (Q.dims == 3) {
                    const float U[2] = {Q.u_min, Q.u_max}, W[2] = {Q.w_min, Q.w_max};
                    for (int c = 0; c < 4; ++c) {
                        s_pts[4 + c][Q.au] = U[c & 1];
                        s_pts[4 + c][Q.aw] = W[c >> 1];
                        s_pts[4 + c][Q.an] = Q.p_n;
                    }
                } else {
                    const float U[2] = {Q.u_min, Q.u_max};
                    for (int c = 0; c < 2; ++c) {
                        s_pts[4 + c][Q.au] = U[c];
                        s_pts[4 + c][Q.an] = Q.p_n;
                        s_pts[4 + c][2] = 0.f;
                    }
                }
            }
        }
        __syncthreads();
        const int item = sm.item;
        if (item >= total_tiles)
            break;
        const int helper = sm.helper;
        const DevRequest &R = s_req;
        const int t = sm.pad;
        const int per_layer = R.tiles_x * R.tiles_y;
        const int layer = t / per_layer;
        const int tt = t - layer * per_layer;
        const int ty = tt / R.tiles_x, tx = tt - ty * R.tiles_x;
        const int ix0 = tx * R.tile_x, ix1 = min(R.nx, ix0 + R.tile_x);
        const int iy0 = ty * R.tile_y, iy1 = min(R.ny, iy0 + R.tile_y);
        const int tw = ix1 - ix0, tn = tw * (iy1 - iy0);
        // row of a tile index vi < 1024 in a row of tw <= 256: the float
        // product is within 1e-6 of vi / tw, whose fraction is 0.5 / tw away
        // from an integer, so the truncation is exact (and cheaper than an
        // integer division)
        const float inv_tw = 1.0f / (float)tw;
        const float zq = R.z_coord[layer];
        const bool want_bits = (R.flags & VCM_EMIT_BITS) && R.bits_out;

        // side of the target plane: s = sn (q_n - p_n) depends on q_n only
        float qn_lo, qn_hi;
        if (R.an == 2) {
            qn_lo = qn_hi = zq;
        } else if (R.an == 0) {
            qn_lo = R.x_coord[ix0]; qn_hi = R.x_coord[ix1 - 1];
        } else {
            qn_lo = R.y_coord[iy0]; qn_hi = R.y_coord[iy1 - 1];
        }
        const bool viewer = (R.flags & VCM_VIEWER) != 0;
        const bool any_front = viewer || (R.flags & VCM_TWO_SIDED) ||
                               (R.sn > 0.f ? (qn_hi - R.p_n > 0.f) : (R.p_n - qn_lo > 0.f));
        if (!CHUNKS && !any_front && !want_bits) {
            for (int i = tid; i < tn; i += kThreads) {
                const int ix = ix0 + i % tw, iy = iy0 + i / tw;
                put_v(R, ((long long)layer * R.ny + iy) * R.nx + ix, 0.f);
            }
            __syncthreads();
            if (tid == 0)
                sm.item = -2;
            continue;
        }

        // Whole-tile shortcut from recorded blockers (launches with the
        // whole-tile check): a box that blocked this tile position on
        // another layer, or a neighbouring position, often blocks this tile
        // too, so threads 0-4 test those first, against the same 16
        // segments as the check below; a tile one of them blocks skips its
        // cull.  Any tile writes the table, so which blocker it keeps is a
        // race; a box counts only if it certainly blocks, so results do not
        // depend on the table.
        bool pre_blocked = false;
        unsigned pre_tests = 0;
        const bool tile_check = TILE_CHECK && !CHUNKS && !viewer;
        if (tile_check && R.blk_base >= 0) {
            int *blockers = work + kWorkHeader + kBlockerOff;
            const int tile_pos = ty * R.tiles_x + tx;
            bool full = false;
            if (warp == 0) {
                // lanes 4c + k: candidate c (this position, then its four
                // neighbours) against corner viewpoint k of the tile
                const int c = lane >> 2, corner = lane & 3;
                int cand = -1;
                bool ok = false;
                if (c < 5) {
                    const int px = tx + (c == 1) - (c == 2), py = ty + (c == 3) - (c == 4);
                    cand = (px >= 0 && px < R.tiles_x && py >= 0 && py < R.tiles_y)
                               ? __ldcg(blockers + R.blk_base + py * R.tiles_x + px)
                               : -1;
                    if (cand >= 0 && cand < sc.n_boxes) {
                        const float4 *gb = sc.boxes[R.perm];
                        // the tile's corners from shared memory at each use, so that
                        // they are not held in registers through the cull
                        const float qx = (corner & 1) ? s_pts[1][0] : s_pts[0][0];
                        const float qy = (corner & 2) ? s_pts[2][1] : s_pts[0][1];
                        const float qu = R.au == 0 ? qx : (R.au == 1 ? qy : zq);
                        const float qn = R.an == 0 ? qx : (R.an == 1 ? qy : zq);
                        const float qw = R.dims == 3 ? (R.aw == 0 ? qx : (R.aw == 1 ? qy : zq)) : 0.f;
                        ok = box_blocks_all(R, __ldg(&gb[2 * cand]), __ldg(&gb[2 * cand + 1]), qu, qn, qw);
                        pre_tests = 4;
                    }
                }
                const unsigned m = __ballot_sync(kFull, ok);
                full = c < 5 && ((m >> (4 * c)) & 0xFu) == 0xFu;
                if (full && corner == 0 && c != 0)
                    blockers[R.blk_base + tile_pos] = cand;
            }
            pre_blocked = __syncthreads_or(full) != 0;
        }

        const int np = (R.dims == 3) ? 8 : 6;
        // candidates past the staged ones: the block's spill region for its
        // own tile, the record's ids in the pool for a chunk
        const int *list_tail = spill;
        if (!CHUNKS && !pre_blocked) {
            hull_planes(R.dims, s_pts, np, sm);
            __syncthreads();
        }
        const int n_planes = min(sm.n_planes, kMaxPlanes);

        // walk the grid cells under the hull's footprint.  In the xy plane
        // the footprint is the convex hull of two axis-aligned rectangles,
        // A (the tile's viewpoints) and B (the target's shadow on the
        // ground plane), which is the union over l in [0, 1] of the
        // rectangles (1 - l) A + l B.  A row of cells meets it for the l whose
        // rectangle reaches the row -- an interval, from two linear
        // inequalities -- and over the x-range those rectangles sweep, which
        // is spanned by the interval's two ends.  Rows are taken 128 at a
        // time: one thread finds a row's span, a block scan lays the spans
        // end to end, and the threads share out the cells.
        if (!CHUNKS && !pre_blocked) {
            float ax0 = s_pts[0][0], ax1 = ax0, ay0 = s_pts[0][1], ay1 = ay0;
            for (int l = 1; l < 4; ++l) {
                ax0 = fminf(ax0, s_pts[l][0]); ax1 = fmaxf(ax1, s_pts[l][0]);
                ay0 = fminf(ay0, s_pts[l][1]); ay1 = fmaxf(ay1, s_pts[l][1]);
            }
            float bx0 = s_pts[4][0], bx1 = bx0, by0 = s_pts[4][1], by1 = by0;
            for (int l = 5; l < np; ++l) {
                bx0 = fminf(bx0, s_pts[l][0]); bx1 = fmaxf(bx1, s_pts[l][0]);
                by0 = fminf(by0, s_pts[l][1]); by1 = fmaxf(by1, s_pts[l][1]);
            }
            // how far a cell's boxes reach past the cell, plus 1 m: far more
            // than the rounding of any quantity below (coordinates are
            // within 2^14 m), so no cell that can hold an occluder is missed
            const float oh = sc.overhang + 1.f;
            const int cy0 = max((int)floorf((fminf(ay0, by0) - oh - sc.gy0) * sc.inv_cell), 0);
            const int cy1 = min((int)floorf((fmaxf(ay1, by1) + oh - sc.gy0) * sc.inv_cell), sc.gny - 1);
            const float dy0 = by0 - ay0, dy1 = by1 - ay1;
            const float4 *world = sc.boxes[0];
            for (int r0 = cy0; r0 <= cy1; r0 += kThreads) {
                const int row = r0 + tid;
                int xa = 0, width = 0;
                if (row <= cy1) {
                    const float ya = fmaf((float)row, sc.cell, sc.gy0) - oh, yb = ya + sc.cell + 2.f * oh;
                    float l0 = 0.f, l1 = 1.f;
                    // lower edge ay0 + l dy0 <= yb
                    if (dy0 > 0.f)
                        l1 = fminf(l1, (yb - ay0) / dy0);
                    else if (dy0 < 0.f)
                        l0 = fmaxf(l0, (yb - ay0) / dy0);
                    else if (ay0 > yb)
                        l1 = -1.f;
                    // upper edge ay1 + l dy1 >= ya
                    if (dy1 > 0.f)
                        l0 = fmaxf(l0, (ya - ay1) / dy1);
                    else if (dy1 < 0.f)
                        l1 = fminf(l1, (ya - ay1) / dy1);
                    else if (ay1 < ya)
                        l1 = -1.f;
                    if (l0 <= l1) {
                        const float xl = fminf(fmaf(l0, bx0 - ax0, ax0), fmaf(l1, bx0 - ax0, ax0));
                        const float xh = fmaxf(fmaf(l0, bx1 - ax1, ax1), fmaf(l1, bx1 - ax1, ax1));
                        const int c0 = max((int)floorf((xl - oh - sc.gx0) * sc.inv_cell), 0);
                        const int c1 = min((int)floorf((xh + oh - sc.gx0) * sc.inv_cell), sc.gnx - 1);
                        if (c1 >= c0) {
                            xa = c0;
                            width = c1 - c0 + 1;
                        }
                    }
                }
                // exclusive scan of the widths over the block
                int incl = width;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int t = __shfl_up_sync(kFull, incl, off);
                    if (lane >= off)
                        incl += t;
                }
                if (lane == 31)
                    s_wsum[warp] = incl;
                __syncthreads();
                int before = 0, total = 0;
#pragma unroll
                for (int w2 = 0; w2 < kWarps; ++w2) {
                    before += w2 < warp ? s_wsum[w2] : 0;
                    total += s_wsum[w2];
                }
                s_rowpre[tid] = before + incl - width;
                s_rowx[tid] = xa;
                __syncthreads();
                // (a) threads over cells: the cells whose bounds meet the
                // hull are listed (box range start and length)
                for (int c = tid; c < total; c += kThreads) {
                    // the row of cell c: the last t with s_rowpre[t] <= c
                    int t = 0;
#pragma unroll
                    for (int step = kThreads / 2; step > 0; step >>= 1)
                        if (s_rowpre[t + step] <= c)
                            t += step;
                    const int cell = (r0 + t) * sc.gnx + s_rowx[t] + (c - s_rowpre[t]);
                    const int b = sc.cell_start[cell], e = sc.cell_start[cell + 1];
                    if (b == e || outside(sm.planes, n_planes, sc.cell_lo[cell], sc.cell_hi[cell]))
                        continue;
                    const int k = atomicAdd(&s_npass, 1);
                    if (k < kPassCap) {
                        s_passb[k] = b;
                        s_passn[k] = e - b;
                        continue;
                    }
                    for (int s = b; s < e; ++s)   // list full: this cell's boxes here
                        add_candidate(world, sm.planes, n_planes, s, sm, s_ids, box_cap, spill, spill_slot, R,
                                      sc.n_boxes);
                }
                __syncthreads();
                // (b) exclusive scan of the listed cells' box counts
                const int n_pass = min(s_npass, kPassCap);
                {
                    int cnt[kPassCap / kThreads], local = 0;
#pragma unroll
                    for (int q = 0; q < kPassCap / kThreads; ++q) {
                        const int k = tid * (kPassCap / kThreads) + q;
                        cnt[q] = k < n_pass ? s_passn[k] : 0;
                        local += cnt[q];
                    }
                    int incl = local;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int t = __shfl_up_sync(kFull, incl, off);
                        if (lane >= off)
                            incl += t;
                    }
                    if (lane == 31)
                        s_wsum2[warp] = incl;
                    __syncthreads();
                    int run = 0, all = 0;
#pragma unroll
                    for (int w2 = 0; w2 < kWarps; ++w2) {
                        run += w2 < warp ? s_wsum2[w2] : 0;
                        all += s_wsum2[w2];
                    }
                    run += incl - local;
#pragma unroll
                    for (int q = 0; q < kPassCap / kThreads; ++q) {
                        const int k = tid * (kPassCap / kThreads) + q;
                        s_passp[k] = k < n_pass ? run : INT_MAX;
                        run += cnt[q];
                    }
                    if (tid == 0)
                        s_passp[kPassCap] = all;
                }
                __syncthreads();
                // (c) threads over the listed cells' boxes
                const int n_boxes_listed = s_passp[kPassCap];
                for (int i = tid; i < n_boxes_listed; i += kThreads) {
                    // the cell of box i: the last k with s_passp[k] <= i
                    int k = 0;
#pragma unroll
                    for (int step = kPassCap / 2; step > 0; step >>= 1)
                        if (s_passp[k + step] <= i)
                            k += step;
                    add_candidate(world, sm.planes, n_planes, s_passb[k] + (i - s_passp[k]), sm, s_ids, box_cap,
                                  spill, spill_slot, R, sc.n_boxes);
                }
                if (tid == 0)
                    s_npass = 0;
                __syncthreads();   // the next rows reuse the span arrays
            }
        } else if (CHUNKS) {
            // a chunk: the owner's candidate list, in the owner's order, and
            // the chunk's viewpoints
            const int *ch = work + kWorkHeader + kChunkOff + (size_t)(2 + kChunkVp) * helper;
            const int *rec = work + kWorkHeader + kRecOff + (size_t)kRecInts * __ldcg(ch);
            const int cnt = __ldcg(rec + 1), n_ch = __ldcg(ch + 1);
            const int *ids = work + kWorkHeader + kPoolOff + __ldcg(rec + 2);
            for (int i = tid; i < min(cnt, box_cap); i += kThreads)
                s_ids[i] = __ldcg(ids + i);
            list_tail = ids + box_cap;
            for (int i = tid; i < n_ch; i += kThreads)
                if (IN_BOUNDS(i, kChunkVp, R.stats))
                    s_und[i] = __ldcg(ch + 2 + i);
            if (tid == 0) {
                sm.count = cnt;
                sm.n_und = n_ch;
            }
        }
        __syncthreads();
        // A block without a spill region (its bounded claim gave up) keeps
        // only the candidates it staged: its request is already flagged
        // (vcm_stats.error), and it reads no region it does not own.
        const int count = spill_slot >= 0 ? sm.count : min(sm.count, box_cap);
        const int n_smem = min(count, box_cap);
        const float4 *gbox = sc.boxes[R.perm];
        // near-first order of the staged candidates: nearby boxes block the
        // most sightlines, so the all-blocked exits come early.  Keys are the
        // squared footprint distance from the tile centre (a positive float,
        // so its bits order like the value) above the sorted box index.
        if (!CHUNKS && n_smem > 1) {
            const float cx = 0.5f * (R.x_coord[ix0] + R.x_coord[ix1 - 1]);
            const float cy = 0.5f * (R.y_coord[iy0] + R.y_coord[iy1 - 1]);
            auto key_of = [&](int i) {
                const int s = s_ids[i];
                const float4 l = world_box_lo(sc, s), h = world_box_hi(sc, s);
                const float dx = 0.5f * (l.x + h.x) - cx, dy = 0.5f * (l.y + h.y) - cy;
                return ((unsigned long long)__float_as_uint(fmaf(dx, dx, dy * dy)) << 32) | (unsigned)s;
            };
            if (n_smem <= 32) {
                // one warp, in registers
                if (warp == 0) {
                    unsigned long long key = lane < n_smem ? key_of(lane) : ~0ull;
#pragma unroll
                    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                        for (int j = k >> 1; j > 0; j >>= 1) {
                            const unsigned long long other = __shfl_xor_sync(kFull, key, j);
                            const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
                            key = keep_min ? (key < other ? key : other) : (key > other ? key : other);
                        }
                    if (lane < n_smem)
                        s_ids[lane] = (int)(key & 0xffffffffu);
                }
            } else {
                // longer lists: a counting sort into distance classes (4 per
                // doubling of the squared distance, 128 classes from 1 m^2),
                // near classes first; order within a class is arbitrary.
                // Results do not depend on the order, only how soon the
                // sweeps stop; this takes 4 barriers where a bitonic sort of
                // 256 keys took 36.
                int *cls_rank = reinterpret_cast<int *>(s_box);   // s_box is free until staging
                int *placed = cls_rank + n_smem;
                for (int i = tid; i < kDistClasses; i += kThreads)
                    s_hist[i] = 0;
                __syncthreads();
                for (int i = tid; i < n_smem; i += kThreads) {
                    const unsigned bits = (unsigned)(key_of(i) >> 32);   // float bits of d^2 >= 0
                    const int c = (int)min((unsigned)(kDistClasses - 1), bits > 0x3f800000u ? (bits - 0x3f800000u) >> 21 : 0u);
                    cls_rank[i] = (c << 24) | atomicAdd(&s_hist[c], 1);
                }
                __syncthreads();
                if (warp == 0) {
                    // exclusive scan of the class counts, kDistClasses / 32 per lane
                    int cnt[kDistClasses / 32], sum = 0;
#pragma unroll
                    for (int q = 0; q < kDistClasses / 32; ++q) {
                        cnt[q] = s_hist[lane * (kDistClasses / 32) + q];
                        sum += cnt[q];
                    }
                    int incl = sum;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int t = __shfl_up_sync(kFull, incl, off);
                        if (lane >= off)
                            incl += t;
                    }
                    int run = incl - sum;
#pragma unroll
                    for (int q = 0; q < kDistClasses / 32; ++q) {
                        s_hist[lane * (kDistClasses / 32) + q] = run;
                        run += cnt[q];
                    }
                }
                __syncthreads();
                for (int i = tid; i < n_smem; i += kThreads) {
                    const int cr = cls_rank[i];
                    placed[s_hist[cr >> 24] + (cr & 0xffffff)] = s_ids[i];
                }
                __syncthreads();
                for (int i = tid; i < n_smem; i += kThreads)
                    s_ids[i] = placed[i];
            }
            __syncthreads();
        }
        for (int i = tid; i < n_smem; i += kThreads) {
            const float4 *src = gbox + 2 * s_ids[i];
            cp_async16(&s_box[2 * i], src);
            cp_async16(&s_box[2 * i + 1], src + 1);
        }
        cp_async_wait_all();
        __syncthreads();

        // sweep: warps take the tile's viewpoints one at a time
        unsigned long long tests = 0, corner_tests = 0;
        unsigned rechecks = 0, shortcuts = 0;
        float vmax = 0.f;

        // Whole-tile check.  For a fixed patch, the viewpoints whose segment
        // to it meets a convex box form a convex set (the box's shadow seen
        // from the patch), so a box that certainly blocks the segments from
        // the tile's four corner viewpoints to an extreme patch centre blocks
        // it from the whole tile rectangle; the one-box argument over the
        // target plane then covers every patch of every viewpoint.  Threads
        // take the nearest candidates, one each, against all 16 segments.
        bool tile_blocked = pre_blocked;
        corner_tests += pre_tests;
        if (tile_check && !pre_blocked) {
            bool full = false;
            if (tid < min(n_smem, kThreads)) {
                full = box_blocks_tile(R, s_box[2 * tid], s_box[2 * tid + 1], s_pts[0][0], s_pts[1][0], s_pts[0][1],
                                       s_pts[2][1], zq);
                corner_tests += 16;
                if (full && R.blk_base >= 0)   // for the tiles of this position and its neighbours
                    work[kWorkHeader + kBlockerOff + R.blk_base + ty * R.tiles_x + tx] = s_ids[tid];
            }
            tile_blocked = __syncthreads_or(full) != 0;
        }
        if (tile_blocked) {
            for (int i = tid; i < tn; i += kThreads) {
                const int ix = ix0 + i % tw, iy = iy0 + i / tw;
                const long long vp = ((long long)layer * R.ny + iy) * R.nx + ix;
                put_v(R, vp, 0.f);
                if (want_bits)
                    for (int wd = 0; wd < R.words; ++wd) {
                        const int rem = R.P - 32 * wd;
                        put_word(R, vp * R.words + wd, rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u));
                    }
            }
            if (tid == 0)
                shortcuts += (unsigned)tn;
        }
        if (!CHUNKS && viewer) {
            // viewer-centric: threads take cells, one segment each
            for (int vi = tid; vi < tn; vi += kThreads) {
                const int ry = (int)(((float)vi + 0.5f) * inv_tw), ix = ix0 + vi - ry * tw, iy = iy0 + ry;
                const long long vp = ((long long)layer * R.ny + iy) * R.nx + ix;
                bool blocked;
                const float v = viewer_cell(R, s_box, n_smem, list_tail, count, gbox, R.x_coord[ix], R.y_coord[iy],
                                            R.dims == 3 ? zq : 0.f, blocked, tests, rechecks, sc.n_boxes);
                put_v(R, vp, v);
                if (want_bits)
                    put_word(R, vp, blocked ? 1u : 0u);
                vmax = fmaxf(vmax, v);
            }
        }
        // First every viewpoint gets the one-box check, four per warp with
        // lanes as 4 viewpoints x the 8 nearest candidates (the blocking box
        // is almost always among them); the viewpoints it leaves open are
        // listed and then taken one per warp for the check over the 32
        // nearest and the separable sweep.
        for (; !CHUNKS && !viewer && !tile_blocked;) {
            int base = 0;
            if (lane == 0)
                base = atomicAdd(&s_next, 4);
            base = __shfl_sync(kFull, base, 0);
            if (base >= tn)
                break;
            const int sub = lane >> 3, bl = lane & 7;
            const int nb8 = min(n_smem, 8);
            {
                const int vi = base + sub;
                long long vp = 0;
                bool active = false, behind = false, full = false;
                if (vi < tn) {
                    const int ry = (int)(((float)vi + 0.5f) * inv_tw), ix = ix0 + vi - ry * tw, iy = iy0 + ry;
                    vp = ((long long)layer * R.ny + iy) * R.nx + ix;
                    const float qx = R.x_coord[ix], qy = R.y_coord[iy];
                    const float qu = R.au == 0 ? qx : (R.au == 1 ? qy : zq);
                    const float qn = R.an == 0 ? qx : (R.an == 1 ? qy : zq);
                    const float qw = R.dims == 3 ? (R.aw == 0 ? qx : (R.aw == 1 ? qy : zq)) : 0.f;
                    active = want_bits || facing(R, qn);
                    behind = !active;
                    if (active && bl < nb8) {
                        full = box_blocks_all(R, s_box[2 * bl], s_box[2 * bl + 1], qu, qn, qw);
                        corner_tests += 4;
                    }
                }
                const unsigned m = __ballot_sync(kFull, full);
                const bool decided = active && ((m >> (8 * sub)) & 0xffu) != 0;
                if (behind && bl == 0)
                    put_v(R, vp, 0.f);   // behind the target
                if (decided) {
                    if (bl == 0) {
                        put_v(R, vp, 0.f);
                        ++shortcuts;
                    }
                    if (want_bits)
                        for (int wd = bl; wd < R.words; wd += 8) {
                            const int rem = R.P - 32 * wd;
                            put_word(R, vp * R.words + wd, rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u));
                        }
                }
                if (active && !decided && bl == 0) {
                    const int at = atomicAdd(&sm.n_und, 1);
                    if (IN_BOUNDS(at, kMaxTileViewpoints, R.stats))
                        s_und[at] = vi;
                }
            }
        }
        __syncthreads();
        int n_und = (viewer || tile_blocked) ? 0 : sm.n_und;
        // Work sharing, first pass (share == 1): a tile with at least
        // R.min_publish open viewpoints publishes them, in chunks of up to
        // R.chunk_vp, with its candidate list (when the list is staged
        // whole), and the second pass sweeps them.  Without it a few hundred
        // tiles of mostly visible viewpoints set the end of the launch (3D
        // workload: 100-290 us each against 17 us for the median tile).  A
        // tile with a list longer than kPublishBoxes publishes only with at
        // least kPublishHeavy open viewpoints (each chunk stages the list
        // again; a spilled list's tail is read from the record), and a tile
        // whose publication would pass a cap of the arena keeps its
        // viewpoints.
        if (!CHUNKS && share == 1 && spill_slot >= 0 && n_und >= R.min_publish &&
            (count <= kPublishBoxes || n_und >= kPublishHeavy)) {
            int *arena = work + kWorkHeader;
            const int cvp = R.chunk_vp;
            if (tid == 0) {
                const int want = (n_und + cvp - 1) / cvp;
                int rec = kRecCap, base = 0, got = 0, off = 0;
                // counters move only while their caps are not reached
                if (__ldcg(work + 1) < kRecCap && __ldcg(work + 4) < kPoolInts && __ldcg(work + 2) < kChunkCap) {
                    rec = atomicAdd(work + 1, 1);
                    if (rec < kRecCap) {
                        off = atomicAdd(work + 4, count);
                        if (off <= kPoolInts - count) {
                            base = atomicAdd(work + 2, want);
                            got = max(0, min(want, kChunkCap - base));
                        }
                    }
                }
                sm.pub[0] = rec;
                sm.pub[1] = base;
                sm.pub[2] = got;
                sm.pub[3] = off;
                s_next2 = min(n_und, got * cvp);   // the tile keeps the rest
                if (got > 0)
                    atomicAdd(&R.stats->shared_viewpoints, (unsigned long long)s_next2);
            }
            __syncthreads();
            const int pub_n = sm.pub[2];
            if (pub_n > 0) {
                const int rec = sm.pub[0], pub_base = sm.pub[1], off = sm.pub[3];
                int *rp = arena + kRecOff + (size_t)kRecInts * rec;
                int *ids = arena + kPoolOff + off;
                if (tid == 0) {
                    rp[0] = item;
                    rp[1] = count;
                    rp[2] = off;
                }
                for (int i = tid; i < count; i += kThreads)
                    ids[i] = i < n_smem ? s_ids[i] : spill[i - n_smem];
                for (int i = tid; i < pub_n * (2 + kChunkVp); i += kThreads) {
                    const int j = i / (2 + kChunkVp), r = i - j * (2 + kChunkVp);
                    const int n_j = min(cvp, n_und - j * cvp);
                    arena[kChunkOff + (size_t)(2 + kChunkVp) * (pub_base + j) + r] =
                        r == 0 ? rec : r == 1 ? n_j : (r - 2 < n_j ? s_und[j * cvp + r - 2] : -1);
                }
            }
        }
        // then the undecided viewpoints, one per warp at a time
        for (;;) {
            int k = 0;
            if (lane == 0)
                k = atomicAdd(&s_next2, 1);
            k = __shfl_sync(kFull, k, 0);
            if (k >= n_und)
                break;
            {
                const int vi = s_und[k];
                const int ry = (int)(((float)vi + 0.5f) * inv_tw), ix = ix0 + vi - ry * tw, iy = iy0 + ry;
                const long long vp = ((long long)layer * R.ny + iy) * R.nx + ix;
                const float qx = R.x_coord[ix], qy = R.y_coord[iy];
                const float qu = R.au == 0 ? qx : (R.au == 1 ? qy : zq);
                const float qn = R.an == 0 ? qx : (R.an == 1 ? qy : zq);
                const float qw = R.dims == 3 ? (R.aw == 0 ? qx : (R.aw == 1 ? qy : zq)) : 0.f;
                const bool front = facing(R, qn);
                if (n_smem > 8) {
                    const int nb_short = min(n_smem, 32);
                    if (lane < nb_short)
                        corner_tests += 4;
                    if (one_box_blocks_all(R, s_box, nb_short, qu, qn, qw)) {
                        if (lane == 0) {
                            put_v(R, vp, 0.f);
                            ++shortcuts;
                        }
                        if (want_bits)
                            for (int wd = lane; wd < R.words; wd += 32) {
                                const int rem = R.P - 32 * wd;
                                put_word(R, vp * R.words + wd, rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u));
                            }
                        continue;
                    }
                }
                // the pyramid filter pays for its set-up only on long candidate lists
                Plane *pyr = s_pyr[warp];
                const bool use_pyr = count > kPyramidMinCount;
                float v;
                if (EXTRA && (R.cone || (R.flags & VCM_TWO_SIDED))) {
                    // sides and cone: one sweep variant of their own (8 rows
                    // per pass; the host sets k_rows = 8 for these requests)
                    v = sweep_viewpoint<8, true>(R, s_box, n_smem, list_tail, count, gbox, qu, qn, qw, front, vp, pyr,
                                                 use_pyr, tests, rechecks, sc.n_boxes);
                } else switch (R.k_rows) {
                case 1: v = sweep_viewpoint<1, false>(R, s_box, n_smem, list_tail, count, gbox, qu, qn, qw, front, vp, pyr, use_pyr, tests, rechecks, sc.n_boxes); break;
                case 2: v = sweep_viewpoint<2, false>(R, s_box, n_smem, list_tail, count, gbox, qu, qn, qw, front, vp, pyr, use_pyr, tests, rechecks, sc.n_boxes); break;
                case 4: v = sweep_viewpoint<4, false>(R, s_box, n_smem, list_tail, count, gbox, qu, qn, qw, front, vp, pyr, use_pyr, tests, rechecks, sc.n_boxes); break;
                default: v = sweep_viewpoint<8, false>(R, s_box, n_smem, list_tail, count, gbox, qu, qn, qw, front, vp, pyr, use_pyr, tests, rechecks, sc.n_boxes); break;
                }
                if (!front)
                    v = 0.f;
                if (lane == 0)
                    put_v(R, vp, v);
                vmax = fmaxf(vmax, v);
            }
        }
        // per-tile counters
        for (int off = 16; off > 0; off >>= 1) {
            tests += __shfl_xor_sync(kFull, tests, off);
            corner_tests += __shfl_xor_sync(kFull, corner_tests, off);
            shortcuts += __shfl_xor_sync(kFull, shortcuts, off);
            vmax = fmaxf(vmax, __shfl_xor_sync(kFull, vmax, off));
        }
        if (lane == 0) {
            atomicMax(&R.stats->vmax_bits, __float_as_uint(vmax));
            if (tests)
                atomicAdd(&R.stats->slab_tests, tests);
            if (corner_tests)
                atomicAdd(&R.stats->corner_tests, corner_tests);
            if (shortcuts)
                atomicAdd(&R.stats->shortcut_viewpoints, (unsigned long long)shortcuts);
        }
        for (int off = 16; off > 0; off >>= 1)
            rechecks += __shfl_xor_sync(kFull, rechecks, off);
        if (lane == 0 && rechecks)
            atomicAdd(&R.stats->rechecked, (unsigned long long)rechecks);
        if (tid == 0) {
            if (!CHUNKS)
                atomicAdd(&R.stats->boxes_listed, (unsigned long long)count);
            sm.item = -2;   // one_tile: the next round exits
        }
        __syncthreads();
    }
    if (one_tile && tid == 0 && spill_slot >= 0)
        atomicExch(&spill_busy[spill_slot], 0);
}

// Launch prologue, in one kernel: the tile queue's counter, every request's
// counters and, for the requests that asked for bits, their occlusion-bit
// buffers (the tile kernel sets bits with atomicOr).
__global__ void k_prologue(const DevRequest *__restrict__ reqs, int n_req, int *__restrict__ work)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nt = (long long)gridDim.x * blockDim.x;
    if (t < 5)
        work[t] = 0;   // next tile, records, chunks published, chunks taken, id-pool ints used
    constexpr int kStatWords = (int)(sizeof(vcm_stats) / sizeof(unsigned));
    for (long long i = t; i < (long long)n_req * kStatWords; i += nt)
        reinterpret_cast<unsigned *>(reqs[i / kStatWords].stats)[i % kStatWords] = 0u;
    for (int r = 0; r < n_req; ++r) {
        const DevRequest &R = reqs[r];
        if (!(R.flags & VCM_EMIT_BITS) || !R.bits_out)
            continue;
        const long long n = (long long)R.nx * R.ny * R.nl * R.words;
        for (long long i = t; i < n; i += nt)
            R.bits_out[i] = 0u;
    }
}

// ---------------------------------------------------------------------------
// recoloring from stored occlusion bits (incremental gaze change)
// ---------------------------------------------------------------------------

// Values of one target-centric request from occlusion bits made earlier
// (R.bits_out is read, not written): no occlusion test, only the sides, the
// field-of-view cone, strictness and the measure.  Two passes, because the
// viewpoints that need a measure cluster in the grid:
//  1. one viewpoint per thread: the side test and the viewpoint's bit words
//     (fully blocked, or in strict mode any patch blocked, gives v = 0);
//     the others are appended to a list;
//  2. one warp per listed viewpoint, lanes over patches, the warp holding
//     the bit words in registers.  The summation follows the tile kernel's:
//     a compensated sum per lane, then a fixed-order butterfly.

__device__ __forceinline__ void recolor_point(const DevRequest &R, long long vp, float &qu, float &qn, float &qw)
{
    const long long nxy = (long long)R.nx * R.ny;
    const int layer = (int)(vp / nxy);
    const long long rem = vp - (long long)layer * nxy;   // nx * ny can pass 2^31
    const int iy = (int)(rem / R.nx), ix = (int)(rem - (long long)iy * R.nx);
    const float qx = R.x_coord[ix], qy = R.y_coord[iy], qz = R.dims == 3 ? R.z_coord[layer] : 0.f;
    qu = R.au == 0 ? qx : (R.au == 1 ? qy : qz);
    qn = R.an == 0 ? qx : (R.an == 1 ? qy : qz);
    qw = R.dims == 3 ? (R.aw == 0 ? qx : (R.aw == 1 ? qy : qz)) : 0.f;
}

__global__ void __launch_bounds__(256) k_recolor_scan(const DevRequest *__restrict__ reqs, int *__restrict__ list,
                                                      int *__restrict__ n_list)
{
    __shared__ DevRequest s_r;
    if (threadIdx.x == 0)
        s_r = reqs[0];
    __syncthreads();
    const DevRequest &R = s_r;
    const int lane = threadIdx.x & 31;
    const long long n = (long long)R.nx * R.ny * R.nl;
    const long long step = (long long)gridDim.x * blockDim.x;
    const bool strict = (R.flags & VCM_STRICT) != 0;
    const unsigned last_mask = (R.P & 31) ? ((1u << (R.P & 31)) - 1u) : 0xffffffffu;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += step) {
        const long long vp = base + lane;
        bool live = false;
        if (vp < n) {
            float qu, qn, qw;
            recolor_point(R, vp, qu, qn, qw);
            if (facing(R, qn)) {
                const uint32_t *words = R.bits_out + vp * R.words;
                bool all_blocked = true, any_blocked = false;
                for (int wd = 0; wd < R.words; ++wd) {
                    const unsigned full = wd == R.words - 1 ? last_mask : 0xffffffffu;
                    const unsigned w = __ldg(&words[wd]) & full;
                    all_blocked &= w == full;
                    any_blocked |= w != 0u;
                }
                live = !all_blocked && !(strict && any_blocked);
            }
            if (!live)
                put_v(R, vp, 0.f);
        }
        const unsigned m = __ballot_sync(kFull, live);
        int at = 0;
        if (lane == 0 && m)
            at = atomicAdd(n_list, __popc(m));
        at = __shfl_sync(kFull, at, 0);
        if (live && IN_BOUNDS(at + __popc(m & ((1u << lane) - 1u)), n, R.stats))
            list[at + __popc(m & ((1u << lane) - 1u))] = (int)vp;
    }
}

__global__ void __launch_bounds__(256) k_recolor_measure(const DevRequest *__restrict__ reqs,
                                                         const int *__restrict__ list, const int *__restrict__ n_list)
{
    __shared__ DevRequest s_r;
    if (threadIdx.x == 0)
        s_r = reqs[0];
    __syncthreads();
    const DevRequest &R = s_r;
    const int lane = threadIdx.x & 31;
    const int n = *n_list;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int du = 32 % R.nu, dw = 32 / R.nu;
    float vmax = 0.f;
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const long long vq = list[i];
        float qu, qn, qw;
        recolor_point(R, vq, qu, qn, qw);
        const uint32_t *words = R.bits_out + vq * R.words;
        const float rn = qn - R.p_n;
        const float m_s = R.measure * ((R.flags & VCM_TWO_SIDED) ? fabsf(rn) : R.sn * rn);
        float sum = 0.f, comp = 0.f;
        int iu = lane % R.nu, iw = lane / R.nu;
        unsigned held = 0u;   // bit words k*32 .. k*32+31 of this viewpoint, one per lane
        for (int j = lane, k = 0; k * 32 < R.P; j += 32, ++k) {
            if ((k & 31) == 0) {
                const int wd = k + lane;
                held = wd < R.words ? __ldg(&words[wd]) : 0u;
            }
            const unsigned w = __shfl_sync(kFull, held, k & 31);
            if (j < R.P) {
                const bool blocked = (w >> lane) & 1u;
                const float ru = qu - __ldg(&R.u_coord[iu]), rw = qw - __ldg(&R.w_coord[iw]);
                if (!blocked && !(R.cone && !in_cone_inline(R, ru, rn, rw))) {
                    const float d2 = fmaf(rw, rw, fmaf(ru, ru, rn * rn));
                    float term;
                    if (R.dims == 3) {
                        const float ir = rsqrtf(d2);
                        term = m_s * (ir * ir * ir);
                    } else {
                        term = m_s / d2;
                    }
                    const float tsum = sum + term;
                    if (fabsf(sum) >= fabsf(term))
                        comp += (sum - tsum) + term;
                    else
                        comp += (term - tsum) + sum;
                    sum = tsum;
                }
            }
            // the lane's next patch: 32 further in row-major order
            iu += du;
            iw += dw;
            if (iu >= R.nu) {
                iu -= R.nu;
                ++iw;
            }
        }
        float v = sum + comp;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            v += __shfl_xor_sync(kFull, v, off);
        if (lane == 0)
            put_v(R, vq, v);
        vmax = fmaxf(vmax, v);
    }
    if (lane == 0 && vmax > 0.f)
        atomicMax(&R.stats->vmax_bits, __float_as_uint(vmax));
}

// ---------------------------------------------------------------------------
// colors
// ---------------------------------------------------------------------------

// Color of one value (Def. 1 normalisation): level 0 for v = 0, else
// 1 + floor((L - 1) v / v_ref) capped at L - 1; `edge` marks a value within
// 1e-5 of an interior bin edge.
__device__ __forceinline__ unsigned char quantise_one(float v, float vref, int L, bool &edge)
{
    unsigned char c = 0;
    edge = false;
    if (v > 0.f && vref > 0.f) {
        const float x = (float)(L - 1) * v / vref;
        const int f = (int)floorf(x);
        c = (unsigned char)(1 + min(L - 2, f));
        const float r = rintf(x);
        edge = r >= 1.f && r <= (float)(L - 2) && fabsf(x - r) <= 1e-5f * x;
    }
    return c;
}

// Four consecutive viewpoints per thread: one 16-byte load of values and one
// 4-byte store of colors when the four belong to one request and both
// addresses are aligned, else one at a time.
__global__ void k_quantise(const DevRequest *__restrict__ reqs, const long long *__restrict__ vp_prefix,
                           int n_req, long long total)
{
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; 4 * g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long i0 = 4 * g;
        int lo_r = 0, hi_r = n_req - 1;
        while (lo_r < hi_r) {
            int mid = (lo_r + hi_r + 1) >> 1;
            if (vp_prefix[mid] <= i0)
                lo_r = mid;
            else
                hi_r = mid - 1;
        }
        const DevRequest &R = reqs[lo_r];
        const long long local0 = i0 - vp_prefix[lo_r];
        const long long n_vp = vp_prefix[lo_r + 1] - vp_prefix[lo_r];
        const float vref = R.v_ref_given > 0.f ? R.v_ref_given : __uint_as_float(R.stats->vmax_bits);
        const int L = R.levels;
        if (local0 == 0)
            R.stats->v_ref = vref;
        const float *vsrc = R.v_out + local0;
        unsigned char *cdst = R.color_out ? R.color_out + local0 : nullptr;
        if (local0 + 4 <= n_vp && (reinterpret_cast<uintptr_t>(vsrc) & 15u) == 0 &&
            (reinterpret_cast<uintptr_t>(cdst) & 3u) == 0) {
            const float4 v4 = *reinterpret_cast<const float4 *>(vsrc);
            bool e0, e1, e2, e3;
            const unsigned c = (unsigned)quantise_one(v4.x, vref, L, e0) |
                               ((unsigned)quantise_one(v4.y, vref, L, e1) << 8) |
                               ((unsigned)quantise_one(v4.z, vref, L, e2) << 16) |
                               ((unsigned)quantise_one(v4.w, vref, L, e3) << 24);
            if (cdst && IN_BOUNDS(local0 + 3, (long long)R.nx * R.ny * R.nl, R.stats))
                *reinterpret_cast<unsigned *>(cdst) = c;
            const unsigned n_edge = (unsigned)e0 + (unsigned)e1 + (unsigned)e2 + (unsigned)e3;
            if (n_edge)   // rare; lanes of one warp may belong to different requests
                atomicAdd(&R.stats->edge_cells, n_edge);
            continue;
        }
        // one at a time: the group's last viewpoints may start the next requests
        for (long long i = i0; i < i0 + 4 && i < total; ++i) {
            while (lo_r + 1 < n_req && vp_prefix[lo_r + 1] <= i)
                ++lo_r;
            const DevRequest &Q = reqs[lo_r];
            const long long local = i - vp_prefix[lo_r];
            const float qref = Q.v_ref_given > 0.f ? Q.v_ref_given : __uint_as_float(Q.stats->vmax_bits);
            bool edge;
            const unsigned char c = quantise_one(Q.v_out[local], qref, Q.levels, edge);
            if (Q.color_out && IN_BOUNDS(local, (long long)Q.nx * Q.ny * Q.nl, Q.stats))
                Q.color_out[local] = c;
            if (edge)
                atomicAdd(&Q.stats->edge_cells, 1u);
            if (local == 0)
                Q.stats->v_ref = qref;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

cudaError_t init_device()
{
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64 && done[dev])
        return cudaSuccess;
    unsigned char tri[56][3];
    int n = 0;
    for (int i = 0; i < 8; ++i)
        for (int j = i + 1; j < 8; ++j)
            for (int k = j + 1; k < 8; ++k) {
                tri[n][0] = (unsigned char)i;
                tri[n][1] = (unsigned char)j;
                tri[n][2] = (unsigned char)k;
                ++n;
            }
    if ((e = cudaMemcpyToSymbol(c_tri, tri, sizeof(tri))) != cudaSuccess)
        return e;
    const void *kernels[6] = {(const void *)k_tiles<false, false, false>, (const void *)k_tiles<true, false, false>,
                              (const void *)k_tiles<false, true, false>,  (const void *)k_tiles<true, true, false>,
                              (const void *)k_tiles<false, false, true>,  (const void *)k_tiles<true, false, true>};
    for (const void *k : kernels)
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)tiles_smem_bytes(kMaxBoxCap))) != cudaSuccess)
            return e;
    if (dev >= 0 && dev < 64)
        done[dev] = true;
    return cudaSuccess;
}

// Scratch for callers that cannot allocate device memory (vcm_compute_static).
// A file-scope __device__ array: every GPU that loads the library holds it
// until the process exits.  Host code must not use the symbol as a pointer;
// it asks the runtime for the array's device address once per device.
static __device__ __align__(256) unsigned char g_static_scratch[VCM_STATIC_SCRATCH_BYTES];

cudaError_t static_scratch(void **ptr, size_t *bytes)
{
    static std::mutex mu;
    static void *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_static_scratch)) != cudaSuccess)
            return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    *bytes = sizeof(g_static_scratch);
    return cudaSuccess;
}

cudaError_t launch_grid_build(const float *d_lo_world, const float *d_hi_world, int n, int dims,
                              float gx0, float gy0, float cell, int gnx, int gny,
                              int *d_cell_of, int *d_count, int *d_cursor, int *d_order,
                              int *d_cell_start, float4 *const *d_perm_boxes, float4 *d_cell_lo,
                              float4 *d_cell_hi, unsigned *d_overhang_bits, cudaStream_t stream)
{
    (void)dims;
    const int n_cells = gnx * gny;
    const int tb = 256;
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_count, 0, sizeof(int) * n_cells, stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_cursor, 0, sizeof(int) * n_cells, stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_overhang_bits, 0, sizeof(unsigned), stream)) != cudaSuccess) return e;
    if (n > 0)
        k_box_cell<<<(n + tb - 1) / tb, tb, 0, stream>>>(d_lo_world, d_hi_world, n, gx0, gy0, 1.0f / cell,
                                                          gnx, gny, d_cell_of, d_count);
    // exclusive scan of the counts; its block sums live in d_cell_lo, which
    // k_cell_bounds writes only at the end (16 bytes per cell, 4 per block sum)
    const int n_scan_blocks = (n_cells + kScanChunk - 1) / kScanChunk;
    if (n_scan_blocks > 1024)
        return cudaErrorInvalidValue;
    int *block_sum = reinterpret_cast<int *>(d_cell_lo);
    k_scan_reduce<<<n_scan_blocks, kScanThreads, 0, stream>>>(d_count, n_cells, block_sum);
    k_scan_top<<<1, 1024, 0, stream>>>(block_sum, n_scan_blocks, n_cells, d_cell_start);
    k_scan_down<<<n_scan_blocks, kScanThreads, 0, stream>>>(d_count, n_cells, block_sum, d_cell_start);
    if (n > 0) {
        k_scatter<<<(n + tb - 1) / tb, tb, 0, stream>>>(d_cell_of, n, d_cell_start, d_cursor, d_order);
        // d_cell_of is free after the scatter: the sort's scratch for large cells
        const int sort_blocks = std::min((n_cells + kScanThreads - 1) / kScanThreads, 152 * 8);
        k_sort_cells<<<sort_blocks, kScanThreads, 0, stream>>>(d_cell_start, n_cells, d_order, d_cell_of);
        PermPtrs pp;
        for (int p = 0; p < 6; ++p)
            pp.p[p] = d_perm_boxes[p];
        k_write_boxes<<<(n + tb - 1) / tb, tb, 0, stream>>>(d_lo_world, d_hi_world, n, d_order, pp);
    }
    k_cell_bounds<<<(n_cells + tb - 1) / tb, tb, 0, stream>>>(d_perm_boxes[0], d_cell_start, gnx, gny,
                                                               gx0, gy0, cell, d_cell_lo, d_cell_hi,
                                                               d_overhang_bits);
    return cudaGetLastError();
}

// Blocks of the chunk pass that fit on one SM (its launch bounds allow 7).
static int chunk_blocks_per_sm(int box_cap, bool extra)
{
    int n = 0;
    auto kernel = extra ? k_tiles<true, false, true> : k_tiles<false, false, true>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, tiles_smem_bytes(box_cap)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

int tiles_blocks_per_sm(int box_cap)
{
    // the tile pass's instantiations share their launch bounds (6 blocks of kThreads)
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tiles<false, false, false>, kThreads,
                                                      tiles_smem_bytes(box_cap)) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_tiles(const DevScene &sc, const DevRequest *d_reqs, const int *d_tile_prefix,
                         int n_req, int total_tiles, int *d_work, int *d_spill, int grid_blocks,
                         int box_cap, bool extra, bool tile_check, cudaStream_t stream, bool one_tile,
                         int *d_spill_busy, bool share, int claim_rounds)
{
    if (claim_rounds < 1 || claim_rounds > kClaimRounds)
        return cudaErrorInvalidValue;
    if (total_tiles <= 0)
        return cudaSuccess;
    if (box_cap < 1 || box_cap > kMaxBoxCap)
        return cudaErrorInvalidValue;
    const size_t smem = tiles_smem_bytes(box_cap);
    const int slots = grid_blocks;   // spill regions: the resident-block bound
    if (one_tile) {
        if (!d_spill_busy)
            return cudaErrorInvalidValue;
        grid_blocks = total_tiles;
    }
    auto kernel = extra ? (tile_check ? k_tiles<true, true, false> : k_tiles<true, false, false>)
                        : (tile_check ? k_tiles<false, true, false> : k_tiles<false, false, false>);
    auto chunks = extra ? k_tiles<true, false, true> : k_tiles<false, false, true>;
    share = share && !one_tile;
    kernel<<<grid_blocks, kThreads, smem, stream>>>(sc, d_reqs, d_tile_prefix, n_req, total_tiles, d_work, d_spill,
                                                    box_cap, one_tile ? 1 : 0, d_spill_busy, slots, share ? 1 : 0,
                                                    claim_rounds);
    if (share) {
        // the second pass: the chunks the first published, on a grid scaled
        // from the tile pass's by the two instantiations' blocks per SM
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
        const int per_tile = tiles_blocks_per_sm(box_cap), per_chunk = chunk_blocks_per_sm(box_cap, extra);
        const int chunk_grid = std::max(1, (int)((long long)grid_blocks * per_chunk / std::max(per_tile, 1)));
        chunks<<<chunk_grid, kThreads, smem, stream>>>(sc, d_reqs, d_tile_prefix, n_req, total_tiles, d_work,
                                                        d_spill, box_cap, 0, d_spill_busy, slots, 2, claim_rounds);
    }
    return cudaGetLastError();
}

cudaError_t launch_prologue(const DevRequest *d_reqs, int n_req, int *d_work, bool any_bits, cudaStream_t stream)
{
    if (n_req <= 0)
        return cudaSuccess;
    // without bits there are only n_req counters to clear
    const int blocks = any_bits ? 152 * 4 : std::max(1, std::min(152, (n_req * 16 + 255) / 256));
    k_prologue<<<blocks, 256, 0, stream>>>(d_reqs, n_req, d_work);
    return cudaGetLastError();
}

cudaError_t launch_quantise(const DevRequest *d_reqs, const long long *d_vp_prefix, int n_req,
                            long long total_vp, cudaStream_t stream)
{
    if (total_vp <= 0)
        return cudaSuccess;
    long long blocks = ((total_vp + 3) / 4 + 255) / 256;   // four viewpoints per thread
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    k_quantise<<<(int)blocks, 256, 0, stream>>>(d_reqs, d_vp_prefix, n_req, total_vp);
    return cudaGetLastError();
}

cudaError_t launch_recolor(const DevRequest *d_req, long long n_vp, int sm_count, int *d_list, int *d_n_list,
                           cudaStream_t stream)
{
    if (n_vp <= 0)
        return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d_n_list, 0, sizeof(int), stream);
    if (e != cudaSuccess)
        return e;
    long long blocks = (n_vp + 255) / 256;
    const long long cap = (long long)std::max(sm_count, 1) * 8;
    if (blocks > cap)
        blocks = cap;
    k_recolor_scan<<<(int)blocks, 256, 0, stream>>>(d_req, d_list, d_n_list);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_recolor_measure<<<(int)cap, 256, 0, stream>>>(d_req, d_list, d_n_list);
    return cudaGetLastError();
}

}  // namespace vcm
