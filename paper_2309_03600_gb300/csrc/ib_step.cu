// Time stepping: fused leapfrog (2D, 3D, batched 2D), staggered
// pressure-velocity (2D), source injection, receiver interpolation, the exact
// discrete adjoint and checkpointed velocity gradients.
//
// Paper: p^{t+1} = 2p^t - p^{t-1} + dt^2 c^2 lap p + dt^2 f (2nd-order
// application section), first-order system with the paper's signs and a
// backward-staggered base stencil (1st-order section), modified operators near
// the boundary ("Reconciliation with the Interior Numerical Discretization"),
// zero Dirichlet outer edges (Examples section).
//
// Every step kernel owns a tile of outputs.  The bulk stencil reads a
// shared-memory copy of the tile and its halo.  The immersed-boundary
// corrections of the tile's rows are stored flattened per tile (output slot,
// source offset, weight) and are added by all threads of the block with
// shared-memory atomics -- a balanced, coalesced gather whatever the number of
// IB rows in the tile.  The update, source injection and masking follow, and
// the tile is written once.
//
// Arithmetic: coefficients (dt^2 c^2 / h^2, dt rho c^2 / h, dt / (rho h)) are
// formed in FP64 and rounded once; the leapfrog update is evaluated as
// p + ((p - p_prev) + Kh * lap) to keep one rounding at the field's magnitude.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ib_common.cuh"

std::vector<double> ib_central_second(int M);
std::vector<double> ib_staggered_first(int M);
ib_status ib_make_bins_ext(const Layout& L, int64_t n, const int64_t* pad, int tx, int ty, int tz, TileBins& b,
                           cudaStream_t s);

#define TRY(x)                          \
    do {                                \
        ib_status st_ = (x);            \
        if (st_ != IB_OK) return st_;   \
    } while (0)

// sampled event timing around one time-step kernel launch
#define PROF_LAUNCH(name, stream, ...)                   \
    do {                                                 \
        ProfToken tk_ = ib_prof_begin((name), (stream)); \
        __VA_ARGS__;                                     \
        ib_prof_end(tk_, (stream));                      \
    } while (0)

template <typename T>
static const char* kname(const char* f32, const char* f64) {
    return sizeof(T) == 8 ? f64 : f32;
}

// flattened corrections of one operator for one tile shape
template <typename T>
struct TileView {
    const int32_t* ptr;    // [ntiles + 1]
    const int32_t* loc;
    const int32_t* src;
    const T* w;
    int64_t ntx;
};

template <typename T>
struct PointSet {          // multilinear weights: 8 corner slots per point
    int n;
    const int64_t* idx;    // padded node
    const T* w;
};

// rows of a small gather table (receiver residual injection in the adjoint)
template <typename T>
struct RowView {
    const int64_t* row_pad;
    const int64_t* row_ptr;
    const int64_t* col;
    const T* w;
    const int32_t* tile_ptr;
    const int32_t* perm;
    int64_t ntx;
};

// Each warp takes chunks of 32 consecutive entries, four chunks at a time so that
// four independent gathers are in flight per thread (surface tiles carry
// thousands of entries and would otherwise serialise on memory latency).
// Entries of one row are contiguous, so a segmented warp sum leaves one
// shared-memory atomic per row segment instead of one per entry.
template <typename T>
__device__ __forceinline__ void seg_add(T* acc, int32_t loc, T val, bool valid, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, val, o);
        int32_t l2 = __shfl_up_sync(0xffffffffu, loc, o);
        if (lane >= o && l2 == loc) val += y;
    }
    const int32_t next = __shfl_down_sync(0xffffffffu, loc, 1);
    if (valid && (lane == 31 || next != loc)) atomicAdd(&acc[loc], val);
}

template <typename T>
__device__ __forceinline__ void add_entries_range(const TileView<T>& v, int32_t e0, int32_t e1, const T* f,
                                                  int64_t origin, T* acc, int tid, int nthr);

template <typename T>
__device__ __forceinline__ void add_entries(const TileView<T>& v, int64_t tile, const T* f, int64_t origin, T* acc,
                                            int tid, int nthr) {
    add_entries_range(v, v.ptr[tile], v.ptr[tile + 1], f, origin, acc, tid, nthr);
}

// entries [e0, e1) of a tile (the range read ahead by the caller)
template <typename T>
__device__ __forceinline__ void add_entries_range(const TileView<T>& v, int32_t e0, int32_t e1, const T* f,
                                                  int64_t origin, T* acc, int tid, int nthr) {
    constexpr int U = 4;
    const int lane = tid & 31;
    const int32_t warp_base = (tid & ~31) * U;
    const int32_t step = nthr * U;
    for (int32_t base = e0 + warp_base; base < e1; base += step) {
        int32_t loc[U];
        T val[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t e = base + u * 32 + lane;
            ok[u] = e < e1;
            loc[u] = ok[u] ? v.loc[e] : -1 - lane;
            val[u] = ok[u] ? v.w[e] * f[origin + v.src[e]] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) seg_add(acc, loc[u], val[u], ok[u], lane);
    }
}

// source terms landing in a 2D tile (or one plane of a 3D tile): sadd[local] += w * wavelet
template <typename T, int TXA, int TYA>
__device__ __forceinline__ void tile_sources(const PointSet<T>& src, T wv, int64_t origin, int64_t px, T* sadd,
                                             int tid) {
    if (tid < 8 * src.n) {
        const int64_t rel = src.idx[tid] - origin;
        if (rel >= 0) {
            const int64_t ly = rel / px, lx = rel - ly * px;
            if (ly < TYA && lx < TXA && src.w[tid] != (T)0) atomicAdd(&sadd[ly * TXA + lx], src.w[tid] * wv);
        }
    }
}

// Receivers gid, gid + stride, ... of this launch (stride = the threads that
// record for this shot), so that every receiver is recorded whatever the grid.
template <typename T>
__device__ __forceinline__ void record_receivers(const PointSet<T>& rec, const T* p, T* traces, int nt, int col,
                                                 int64_t gid, int64_t stride) {
    if (col < 0) return;
    for (int64_t r = gid; r < rec.n; r += stride) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) s += rec.w[8 * r + c] * p[rec.idx[8 * r + c]];
        traces[r * nt + col] = s;
    }
}

__device__ __forceinline__ int64_t launch_threads() {
    return (int64_t)gridDim.x * gridDim.y * gridDim.z * blockDim.x * blockDim.y * blockDim.z;
}

// ---------------------------------------------------------------------------
// second-order leapfrog
// ---------------------------------------------------------------------------
template <typename T>
struct StepArgs {
    Layout L;
    T w2[5];             // central 2nd-derivative weights w[0..H]
    const T* p;          // p^n
    const T* pm;         // p^{n-1}
    T* out;              // p^{n+1} (may alias pm)
    const T* Kh;         // dt^2 c^2 / h^2 (0 outside the domain)
    TileView<T> op;
    PointSet<T> src;     // weights include dt^2 / h^d
    const T* wavelet;
    int step;
    PointSet<T> rec;     // receivers sampled from p (the previous step's output)
    T* traces;
    int nt;
    int rec_step;        // trace column written from p (-1: none)
    // batched runs: the two wavefield buffers (p^n is buf[step & 1])
    T* buf0;
    T* buf1;
    int64_t ntx;         // tiles along x
    int64_t ntiles;      // tiles of the shot (blocks beyond only record receivers)
    int dw;              // absorbing layer width in nodes (0: none)
    T da;                // its largest a = eta_max dt / 2
};

// Absorbing layer along the side edges and the bottom (not the top, where the
// immersed boundary is): a = a_max min(1, d^2 / W^2) with d the node's distance
// into the layer of W nodes, d^2 = dx^2 (+ dy^2) + dz^2, dz counted from the
// bottom only.  The damped leapfrog step of p_tt + 2 a / dt p_t = c^2 lap p + f,
//   p^{n+1} = (2 p^n - (1 - a) p^{n-1} + dt^2 c^2 L p^n + dt^2 f) / (1 + a),
// is the undamped update u followed by u - g (u - p^{n-1}) with g = a / (1 + a).
template <typename T>
__device__ __forceinline__ T damp_a(const Layout& L, int dw, T da, int64_t x, int64_t y, int64_t z) {
    const int64_t w = dw;
    const int64_t dx = max(max(w - x, x - (L.nx - 1 - w)), (int64_t)0);
    const int64_t dy = L.ndim == 3 ? max(max(w - y, y - (L.ny - 1 - w)), (int64_t)0) : 0;
    const int64_t dz = max(z - (L.nz - 1 - w), (int64_t)0);
    const int64_t d2 = dx * dx + dy * dy + dz * dz;
    if (d2 == 0) return (T)0;
    const T r = (T)d2 / (T)(w * w);
    return da * (r < (T)1 ? r : (T)1);
}
// does the box [x0, x1] x [y0, y1] x [.., z1] reach into the layer (dw > 0)?
__device__ __forceinline__ bool damp_box(const Layout& L, int dw, int64_t x0, int64_t x1, int64_t y0, int64_t y1,
                                         int64_t z1) {
    return dw > 0 && (x0 < dw || x1 > L.nx - 1 - dw || z1 > L.nz - 1 - dw ||
                      (L.ndim == 3 && (y0 < dw || y1 > L.ny - 1 - dw)));
}
template <typename T>
__device__ __forceinline__ T damp_g(const Layout& L, int dw, T da, int64_t x, int64_t y, int64_t z) {
    const T av = damp_a<T>(L, dw, da, x, y, z);
    return av / ((T)1 + av);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// rounded arithmetic that the compiler may not contract into FMAs
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

// asynchronous global -> shared copy of B bytes (zero fill when !valid)
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(B),
                 "r"(valid ? B : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, int H, int TX, int TZ>
__device__ __forceinline__ void leap2d_tile(const StepArgs<T>& a, int64_t bx, int64_t bz, T (*tile)[TX + 2 * H],
                                            T* acc, T* sadd) {
    static_assert((TZ * TX) % 256 == 0, "whole points per thread");
    constexpr int PT = TZ * TX / 256;
    const int tid = threadIdx.x;
    const int64_t x0 = bx * TX, z0 = bz * TZ;
    const Layout& L = a.L;
    // the halo tile arrives by cp.async (zero fill past the padded array) ...
    for (int i = tid; i < (TZ + 2 * H) * (TX + 2 * H); i += 256) {
        const int lz = i / (TX + 2 * H), lx = i - lz * (TX + 2 * H);
        const int64_t x = x0 + lx - H, z = z0 + lz - H;
        const bool ok = x < L.nx + H && z < L.nz + H;
        cp_async<(int)sizeof(T)>(&tile[lz][lx], ok ? a.p + L.base + z * L.px + x : a.p, ok);
    }
    cp_async_commit();
    for (int i = tid; i < TZ * TX; i += 256) sadd[i] = (T)0;
    // ... while this thread's p_prev and K, and the tile's correction range, load
    const int64_t origin = L.base + z0 * L.px + x0;
    T pmv[PT], khv[PT];
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j, lz = i / TX, lx = i - lz * TX;
        const bool in = x0 + lx < L.nx && z0 + lz < L.nz;
        const int64_t q = origin + lz * L.px + lx;
        pmv[j] = in ? a.pm[q] : (T)0;
        khv[j] = in ? a.Kh[q] : (T)0;
    }
    int32_t e0 = 0, e1 = 0;
    if (a.op.ptr) {
        e0 = a.op.ptr[bz * a.op.ntx + bx];
        e1 = a.op.ptr[bz * a.op.ntx + bx + 1];
    }
    cp_async_wait_all();
    __syncthreads();
    // Laplacian in difference form, sum_k w_k sum_axes (p_{+k} - p_0 + p_{-k} - p_0): the
    // discrete operator annihilates constants exactly in floating point (row sum zero)
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        T c = tile[lz + H][lx + H];
        T s = 0;
#pragma unroll
        for (int k = 1; k <= H; ++k)
            s += a.w2[k] * (((tile[lz + H][lx + H + k] - c) + (tile[lz + H][lx + H - k] - c)) +
                            ((tile[lz + H + k][lx + H] - c) + (tile[lz + H - k][lx + H] - c)));
        acc[i] = s;
    }
    const T wv = a.src.n ? a.wavelet[a.step] : (T)0;
    tile_sources<T, TX, TZ>(a.src, wv, origin, L.px, sadd, tid);
    __syncthreads();
    if (e1 > e0) add_entries_range(a.op, e0, e1, a.p, origin, acc, tid, 256);
    __syncthreads();
    const bool damped = damp_box(L, a.dw, x0, x0 + TX - 1, 0, 0, z0 + TZ - 1);
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j, lz = i / TX, lx = i - lz * TX;
        if (x0 + lx >= L.nx || z0 + lz >= L.nz) continue;
        const int64_t q = origin + lz * L.px + lx;
        const T c = tile[lz + H][lx + H];
        T u = c + ((c - pmv[j]) + khv[j] * acc[i]) + sadd[i];
        if (damped) u -= damp_g<T>(L, a.dw, a.da, x0 + lx, 0, z0 + lz) * (u - pmv[j]);
        a.out[q] = u;
    }
}

template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256) k_leap2d(StepArgs<T> a) {
    __shared__ T tile[TZ + 2 * H][TX + 2 * H];
    __shared__ T acc[TZ * TX];
    __shared__ T sadd[TZ * TX];
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, blk * 256 + threadIdx.x, launch_threads());
    leap2d_tile<T, H, TX, TZ>(a, blockIdx.x, blockIdx.y, tile, acc, sadd);
}

// many shots in one launch: block -> (shot, tile) through the per-shot tile offsets
template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256) k_leap2d_batch(const StepArgs<T>* __restrict__ shots,
                                                      const int64_t* __restrict__ tile0,
                                                      const int32_t* __restrict__ shot_of, int nshot, int step) {
    __shared__ T tile[TZ + 2 * H][TX + 2 * H];
    __shared__ T acc[TZ * TX];
    __shared__ T sadd[TZ * TX];
    const int64_t b = blockIdx.x;
    const int lo = shot_of[b];            // the shot whose tiles include block b
    StepArgs<T> a = shots[lo];
    const int64_t local = b - tile0[lo];
    T* cur = (step & 1) ? a.buf1 : a.buf0;
    T* prev = (step & 1) ? a.buf0 : a.buf1;
    a.p = cur;
    a.pm = prev;
    a.out = prev;
    a.step = step;
    a.rec_step = step - 1;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, local * 256 + threadIdx.x,
                     (tile0[lo + 1] - tile0[lo]) * 256);
    if (local >= a.ntiles) return;   // uniform per block
    leap2d_tile<T, H, TX, TZ>(a, local % a.ntx, local / a.ntx, tile, acc, sadd);
}

template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// A strip 64 wide and up to NSUB tiles of 64 x 8 deep, marched in z with D tiles
// in flight.  Everything a tile reads arrives by 16-byte cp.async: the strip's
// rows of p (columns x0-4 .. x0+67; x0-4 is a multiple of 4 because the row pitch
// is a multiple of 32) into a buffer that holds the whole strip, p_prev and K into
// D+1 stages.  Each thread owns two vertically adjacent points of every tile and
// walks a pointer down its column, so the stencil's shared-memory offsets are
// immediates.  Arithmetic per point is that of leap2d_tile.
template <int H, int NSUB, int D>
struct Strip2D {
    static constexpr int TX = 64, TZ = 8, W = TX + 8, CH = W / 4, ROWS = NSUB * TZ + 2 * H;
    static_assert(H <= 4 && TZ * CH <= 256 && 2 * H <= TZ, "one chunk per thread and tile");
    float rows[ROWS][W];   // row j holds z = zs - H + j
    float pm[D + 1][TZ * TX];
    float kh[D + 1][TZ * TX];
    float acc[TZ * TX];
    float sadd[TZ * TX];
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

template <int H, int NSUB, int D>
__device__ __forceinline__ void leap2d_strip(const StepArgs<float>& a, int64_t bx, int64_t bzc,
                                             Strip2D<H, NSUB, D>& sm) {
    using S = Strip2D<H, NSUB, D>;
    constexpr int TX = S::TX, TZ = S::TZ, W = S::W, CH = S::CH;
    const int tid = threadIdx.x;
    const Layout& L = a.L;
    const int64_t ntz = (L.nz + TZ - 1) / TZ;
    const int64_t bz0 = bzc * NSUB;
    const int nsub = (int)(ntz - bz0 < NSUB ? ntz - bz0 : NSUB);
    const int64_t x0 = bx * TX, zs = bz0 * TZ;
    const int64_t tstep = TZ * L.px;   // elements from one tile's rows to the next
    // This thread's copies: chunk (pr, pc) of each tile's new rows of p (tid < TZ * CH)
    // and chunk (qr, qc) of p_prev (tid < 128) or K (tid >= 128).  A chunk is zero-filled
    // when its row is past the last row a stored point reads, or when it would end past
    // the allocation; it feeds no stored point then.  The chunks move down tstep
    // elements per tile: their offsets, rows and shared addresses are carried along.
    const int pr = tid / CH, pc = tid - pr * CH;
    const bool pcopy = tid < TZ * CH;
    auto copy_row = [&](int j) {   // strip row j (tile 0 only)
        const int64_t z = zs - H + j;
        const int64_t q = (z + H + 1) * L.px + x0 - 4 + 4 * pc;
        const bool ok = z < L.nz + H && q + 4 <= L.total;
        cp_async16(smem_u32(&sm.rows[j][4 * pc]), ok ? a.p + q : a.p, ok);
    };
    int64_t pq = (zs + TZ + 2 * H + pr + 1) * L.px + x0 - 4 + 4 * pc;   // tile 1: strip row TZ + 2H + pr
    const int nzh = (int)(L.nz + H), nzi = (int)L.nz;   // row limits (2D rows < 2^31)
    const int64_t qlim = L.total - 4;                 // last chunk start inside the allocation
    int pz = (int)(zs + TZ + H + pr);
    uint32_t pdst = smem_u32(&sm.rows[0][0]) + 4u * (uint32_t)((TZ + 2 * H + pr) * W + 4 * pc);
    const int qr = (tid & 127) >> 4, qc = tid & 15;
    const float* qsrc = tid < 128 ? a.pm : a.Kh;
    int64_t qq = (zs + qr + H + 1) * L.px + x0 + 4 * qc;                // tile 0
    int qz = (int)(zs + qr);
    const uint32_t qdst0 = smem_u32((tid < 128 ? &sm.pm[0][0] : &sm.kh[0][0]) + qr * TX + 4 * qc);
    int qst = 0;
    // group t (issued in order t = 0, 1, ...): tile t's new rows of p (rows 0 .. TZ + 2H - 1
    // for t = 0), its p_prev and K
    auto issue = [&](int t) {
        if (t < nsub) {
            if (pcopy) {
                if (t == 0) {
                    copy_row(pr);
                    if (pr < 2 * H) copy_row(pr + TZ);
                } else {
                    const bool ok = pz < nzh && pq <= qlim;
                    cp_async16(pdst, ok ? a.p + pq : a.p, ok);
                    pq += tstep;
                    pz += TZ;
                    pdst += 4u * TZ * W;
                }
            }
            const bool ok = qz < nzi && qq <= qlim;
            cp_async16(qdst0 + 4u * TZ * TX * qst, ok ? qsrc + qq : qsrc, ok);
            qq += tstep;
            qz += TZ;
            qst = qst == D ? 0 : qst + 1;
        }
        cp_async_commit();   // empty groups keep the count uniform
    };
    const int lx = tid & (TX - 1), lz0 = 2 * (tid >> 6);
    const int i0 = lz0 * TX + lx;
    sm.sadd[i0] = 0.f;
    sm.sadd[i0 + TX] = 0.f;
#pragma unroll
    for (int t = 0; t < D; ++t) issue(t);
    // this thread's source corner (tid < 8 n) as (row, column) from the strip origin
    int srow = -1, scol = 0;
    float sw = 0.f;
    const float wv = a.src.n ? a.wavelet[a.step] : 0.f;
    if (tid < 8 * a.src.n) {
        const int64_t rel = a.src.idx[tid] - (L.base + zs * L.px + x0);
        if (rel >= 0) {
            const int64_t r = rel / L.px, c = rel - r * L.px;
            if (r < NSUB * TZ && c < TX && a.src.w[tid] != 0.f) {
                srow = (int)r;
                scol = (int)c;
                sw = a.src.w[tid] * wv;
            }
        }
    }
    const int32_t* pp = a.op.ptr ? a.op.ptr + bz0 * a.op.ntx + bx : nullptr;   // tile s's entry range
    int32_t e0 = 0, e1 = 0;
    if (pp) {
        e0 = pp[0];
        e1 = pp[1];
    }
    const float* colp = &sm.rows[lz0][lx + 4];   // this thread's column, tile s
    const bool xin = x0 + lx < L.nx;
    const int zleft = nzi - (int)zs - lz0;       // rows of this thread's column left to store
    float* outp = a.out + (zs + lz0 + H + 1) * L.px + x0 + lx;
    int64_t origin = L.base + zs * L.px + x0;    // tile s
    int st = 0;                                   // stage of tile s
#pragma unroll 1
    for (int s = 0; s < nsub; ++s) {
        cp_async_wait_group<D - 1>();
        __syncthreads();   // tile s has landed; tile s - 1 is done with its buffers
        issue(s + D);
        int32_t f0 = 0, f1 = 0;
        if (s + 1 < nsub && pp) {
            pp += a.op.ntx;
            f0 = pp[0];
            f1 = pp[1];
        }
        // rows z0 + lz0 - H .. z0 + lz0 + 1 + H of this thread's column
        float v[2 * H + 2];
#pragma unroll
        for (int m = 0; m < 2 * H + 2; ++m) v[m] = colp[m * W];
        float cv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float* r0 = colp + (H + j) * W;
            const float c = v[H + j];
            float sum = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k)
                sum += a.w2[k] * (((r0[k] - c) + (r0[-k] - c)) + ((v[H + j + k] - c) + (v[H + j - k] - c)));
            sm.acc[i0 + j * TX] = sum;
            cv[j] = c;
        }
        {
            const int ly = srow - s * TZ;
            if (srow >= 0 && ly >= 0 && ly < TZ) atomicAdd(&sm.sadd[ly * TX + scol], sw);
        }
        __syncthreads();
        if (e1 > e0) {
            add_entries_range(a.op, e0, e1, a.p, origin, sm.acc, tid, 256);
            __syncthreads();
        }
        const float* pmS = sm.pm[st];
        const float* khS = sm.kh[st];
        const bool damped = damp_box(L, a.dw, x0, x0 + TX - 1, 0, 0, zs + (s + 1) * TZ - 1);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int i = i0 + j * TX;
            if (xin && s * TZ + j < zleft) {
                const float c = cv[j];
                float u = c + ((c - pmS[i]) + khS[i] * sm.acc[i]) + sm.sadd[i];
                if (damped) u -= damp_g<float>(L, a.dw, a.da, x0 + lx, 0, zs + s * TZ + lz0 + j) * (u - pmS[i]);
                outp[j * L.px] = u;
            }
            sm.sadd[i] = 0.f;
        }
        e0 = f0;
        e1 = f1;
        colp += TZ * W;
        outp += tstep;
        origin += tstep;
        st = st == D ? 0 : st + 1;
    }
    cp_async_wait_group<0>();   // the empty groups past the strip's end
}

// many shots in one launch, each block a z-marched strip (leap2d_strip)
template <int H, int NSUB, int D, int MINB>
__global__ void __launch_bounds__(256, MINB) k_leap2d_batch_m(const StepArgs<float>* __restrict__ shots,
                                                              const int64_t* __restrict__ tile0,
                                                              const int32_t* __restrict__ shot_of, int nshot,
                                                              int step) {
    __shared__ __align__(16) Strip2D<H, NSUB, D> sm;
    const int64_t b = blockIdx.x;
    const int lo = shot_of[b];
    StepArgs<float> a = shots[lo];
    const int64_t local = b - tile0[lo];
    float* cur = (step & 1) ? a.buf1 : a.buf0;
    float* prev = (step & 1) ? a.buf0 : a.buf1;
    a.p = cur;
    a.pm = prev;
    a.out = prev;
    a.step = step;
    a.rec_step = step - 1;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, local * 256 + threadIdx.x,
                     (tile0[lo + 1] - tile0[lo]) * 256);
    if (local >= a.ntiles) return;   // uniform per block
    leap2d_strip<H, NSUB, D>(a, local % a.ntx, local / a.ntx, sm);
}

// one shot, FP32: block (x, y) is the z-marched strip of column x and chunk y
template <int H, int NSUB, int D>
__global__ void __launch_bounds__(256, 4) k_leap2d_m(StepArgs<float> a) {
    __shared__ __align__(16) Strip2D<H, NSUB, D> sm;
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, blk * 256 + threadIdx.x, launch_threads());
    leap2d_strip<H, NSUB, D>(a, blockIdx.x, blockIdx.y, sm);
}

// ---------------------------------------------------------------------------
// Strips of 64 x 16 tiles with four points per thread (two x-adjacent columns
// of two rows): the z-marched strip of leap2d_strip with the x-pair layout of
// the 3D step.  Per tile a thread loads its two columns' 2H + 2 rows as 8-byte
// pairs and each of its rows' x neighbours (-4 .. +5) in five 8-byte loads, and
// the copy issue, waits, barriers and epilogue serve four points.  The strip is
// NSUB tiles deep and held whole in shared memory; D tiles are in flight.  The
// arithmetic per point is that of leap2d_tile.
// ---------------------------------------------------------------------------
template <int H, int NSUB, int D>
struct Strip4 {
    static constexpr int TX = 64, TZ = 16, W = TX + 8, CH = W / 4, ROWS = NSUB * TZ + 2 * H;
    static constexpr int STAGE = TZ * TX;
    // floats: rows, p_prev and K stages, acc, sadd
    static constexpr size_t FLOATS = (size_t)ROWS * W + 2 * (D + 1) * STAGE + 2 * STAGE;
    static_assert(H <= 4 && 2 * H <= TZ, "x halo of 4 and one tile of look-ahead rows");
};

template <int H, int NSUB, int D>
__device__ __forceinline__ void leap2d_strip4(const StepArgs<float>& a, int64_t bx, int64_t bzc, float* smem) {
    using S = Strip4<H, NSUB, D>;
    constexpr int TX = S::TX, TZ = S::TZ, W = S::W, CH = S::CH, STAGE = S::STAGE;
    float* rows = smem;                                  // [ROWS][W], row j <-> z = zs - H + j
    float* pm = rows + S::ROWS * W;                      // [D + 1][STAGE]
    float* kh = pm + (D + 1) * STAGE;                    // [D + 1][STAGE]
    float* acc = kh + (D + 1) * STAGE;                   // [STAGE]
    float* sadd = acc + STAGE;                           // [STAGE]
    const int tid = threadIdx.x;
    const Layout& L = a.L;
    const int64_t ntz = (L.nz + TZ - 1) / TZ;
    const int64_t bz0 = bzc * NSUB;
    const int nsub = (int)(ntz - bz0 < NSUB ? ntz - bz0 : NSUB);
    const int64_t x0 = bx * TX, zs = bz0 * TZ;
    const int64_t qlim = L.total - 4;
    // copies of tile t: its new rows of p (all TZ + 2H rows for t = 0), and its
    // p_prev and K (chunk tid of each: row tid >> 4, columns 4 (tid & 15) ..)
    auto issue = [&](int t) {
        if (t < nsub) {
            const int j0 = t == 0 ? 0 : t * TZ + 2 * H;           // first strip row to fetch
            const int nr = t == 0 ? TZ + 2 * H : TZ;
            for (int c = tid; c < nr * CH; c += 256) {
                const int r = c / CH, pc = c - r * CH;
                const int j = j0 + r;
                const int64_t z = zs - H + j;
                const int64_t q = (z + H + 1) * L.px + x0 - 4 + 4 * pc;
                const bool ok = z < L.nz + H && q <= qlim;
                cp_async16(smem_u32(rows + j * W + 4 * pc), ok ? a.p + q : a.p, ok);
            }
            const int st = t % (D + 1);
            const int qr = tid >> 4, qc = tid & 15;
            const int64_t z = zs + (int64_t)t * TZ + qr;
            const int64_t q = (z + H + 1) * L.px + x0 + 4 * qc;
            const bool ok = z < L.nz && q <= qlim;
            cp_async16(smem_u32(pm + st * STAGE + qr * TX + 4 * qc), ok ? a.pm + q : a.pm, ok);
            cp_async16(smem_u32(kh + st * STAGE + qr * TX + 4 * qc), ok ? a.Kh + q : a.Kh, ok);
        }
        cp_async_commit();   // empty groups keep the count uniform
    };
    const int cx = tid & 31, rz = tid >> 5;
    const int lx = 2 * cx, lz0 = 2 * rz;                // points (lz0 + j, lx + k), j, k in {0, 1}
    const int i0 = lz0 * TX + lx;
    *reinterpret_cast<float2*>(sadd + i0) = make_float2(0.f, 0.f);
    *reinterpret_cast<float2*>(sadd + i0 + TX) = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < D; ++t) issue(t);
    int srow = -1, scol = 0;
    float sw = 0.f;
    const float wv = a.src.n ? a.wavelet[a.step] : 0.f;
    if (tid < 8 * a.src.n) {
        const int64_t rel = a.src.idx[tid] - (L.base + zs * L.px + x0);
        if (rel >= 0) {
            const int64_t r = rel / L.px, c = rel - r * L.px;
            if (r < NSUB * TZ && c < TX && a.src.w[tid] != 0.f) {
                srow = (int)r;
                scol = (int)c;
                sw = a.src.w[tid] * wv;
            }
        }
    }
    const int32_t* pp = a.op.ptr ? a.op.ptr + bz0 * a.op.ntx + bx : nullptr;
    int32_t e0 = 0, e1 = 0;
    if (pp) {
        e0 = pp[0];
        e1 = pp[1];
    }
    const float* colp = rows + lz0 * W + lx + 4;        // this thread's column pair, tile s
    const bool xa = x0 + lx < L.nx, xb = x0 + lx + 1 < L.nx;
    const int zleft = (int)(L.nz - zs) - lz0;           // rows of this thread left to store
    float* outp = a.out + (zs + lz0 + H + 1) * L.px + x0 + lx;
    int64_t origin = L.base + zs * L.px + x0;
#pragma unroll 1
    for (int s = 0; s < nsub; ++s) {
        cp_async_wait_group<D - 1>();
        __syncthreads();   // tile s has landed; tile s - 1 is done with its buffers
        issue(s + D);
        int32_t f0 = 0, f1 = 0;
        if (s + 1 < nsub && pp) {
            pp += a.op.ntx;
            f0 = pp[0];
            f1 = pp[1];
        }
        float2 v[2 * H + 2];   // rows lz0 - H .. lz0 + 1 + H of the two columns
#pragma unroll
        for (int m = 0; m < 2 * H + 2; ++m) v[m] = *reinterpret_cast<const float2*>(colp + m * W);
        float2 cv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float* r0 = colp + (H + j) * W;
            float2 xr[5];   // r0[-4 .. 5]
#pragma unroll
            for (int i = 0; i < 5; ++i) xr[i] = *reinterpret_cast<const float2*>(r0 + 2 * i - 4);
            auto X = [&](int o) -> float {
                const int i = o + 4;
                return (i & 1) ? xr[i >> 1].y : xr[i >> 1].x;
            };
            const float ca = v[H + j].x, cb = v[H + j].y;
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                sa += a.w2[k] * (((X(k) - ca) + (X(-k) - ca)) + ((v[H + j + k].x - ca) + (v[H + j - k].x - ca)));
                sb += a.w2[k] * (((X(1 + k) - cb) + (X(1 - k) - cb)) + ((v[H + j + k].y - cb) + (v[H + j - k].y - cb)));
            }
            *reinterpret_cast<float2*>(acc + i0 + j * TX) = make_float2(sa, sb);
            cv[j] = make_float2(ca, cb);
        }
        {
            const int ly = srow - s * TZ;
            if (srow >= 0 && ly >= 0 && ly < TZ) atomicAdd(&sadd[ly * TX + scol], sw);
        }
        __syncthreads();
        if (e1 > e0) {
            add_entries_range(a.op, e0, e1, a.p, origin, acc, tid, 256);
            __syncthreads();
        }
        const int st = s % (D + 1);
        const float* pmS = pm + st * STAGE;
        const float* khS = kh + st * STAGE;
        const bool damped = damp_box(L, a.dw, x0, x0 + TX - 1, 0, 0, zs + (s + 1) * TZ - 1);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int i = i0 + j * TX;
            const float2 pmv = *reinterpret_cast<const float2*>(pmS + i);
            const float2 khv = *reinterpret_cast<const float2*>(khS + i);
            const float2 ac = *reinterpret_cast<const float2*>(acc + i);
            const float2 sd = *reinterpret_cast<const float2*>(sadd + i);
            const float c0 = cv[j].x, c1 = cv[j].y;
            float u0 = c0 + ((c0 - pmv.x) + khv.x * ac.x) + sd.x;
            float u1 = c1 + ((c1 - pmv.y) + khv.y * ac.y) + sd.y;
            if (damped) {
                const int64_t z = zs + s * TZ + lz0 + j;
                u0 -= damp_g<float>(L, a.dw, a.da, x0 + lx, 0, z) * (u0 - pmv.x);
                u1 -= damp_g<float>(L, a.dw, a.da, x0 + lx + 1, 0, z) * (u1 - pmv.y);
            }
            if (s * TZ + j < zleft) {
                if (xb) *reinterpret_cast<float2*>(outp + j * L.px) = make_float2(u0, u1);
                else if (xa) outp[j * L.px] = u0;
            }
            *reinterpret_cast<float2*>(sadd + i) = make_float2(0.f, 0.f);
        }
        e0 = f0;
        e1 = f1;
        colp += TZ * W;
        outp += TZ * L.px;
        origin += TZ * L.px;
    }
    cp_async_wait_group<0>();   // the empty groups past the strip's end
}

// many shots in one launch, each block a z-marched strip of 64 x 16 tiles
template <int H, int NSUB, int D, int MINB>
__global__ void __launch_bounds__(256, MINB) k_leap2d_batch_m4(const StepArgs<float>* __restrict__ shots,
                                                               const int64_t* __restrict__ tile0,
                                                               const int32_t* __restrict__ shot_of, int nshot,
                                                               int step) {
    extern __shared__ __align__(16) float strip4_sm[];
    const int64_t b = blockIdx.x;
    const int lo = shot_of[b];
    StepArgs<float> a = shots[lo];
    const int64_t local = b - tile0[lo];
    float* cur = (step & 1) ? a.buf1 : a.buf0;
    float* prev = (step & 1) ? a.buf0 : a.buf1;
    a.p = cur;
    a.pm = prev;
    a.out = prev;
    a.step = step;
    a.rec_step = step - 1;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, local * 256 + threadIdx.x,
                     (tile0[lo + 1] - tile0[lo]) * 256);
    if (local >= a.ntiles) return;   // uniform per block
    leap2d_strip4<H, NSUB, D>(a, local % a.ntx, local / a.ntx, strip4_sm);
}

// one shot, FP32: block (x, y) is the z-marched strip of column x and chunk y
template <int H, int NSUB, int D>
__global__ void __launch_bounds__(256, 3) k_leap2d_m4(StepArgs<float> a) {
    extern __shared__ __align__(16) float strip4_sm[];
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, blk * 256 + threadIdx.x, launch_threads());
    leap2d_strip4<H, NSUB, D>(a, blockIdx.x, blockIdx.y, strip4_sm);
}

// Batched recompute step n of a checkpoint segment, on z-marched strips: the
// shot's segment buffer (buf0) holds p^{c-1+j} in slot j, and step n = c + j
// writes slot j + 2.  The block map counts strips, ntx * ceil(ceil(nz / 8) / NSUB)
// per shot.
template <int H, int NSUB, int D>
__global__ void __launch_bounds__(256, 4) k_leap2d_batch_seg_m(const StepArgs<float>* __restrict__ shots,
                                                               const int64_t* __restrict__ tile0,
                                                               const int32_t* __restrict__ shot_of, int n, int j) {
    __shared__ __align__(16) Strip2D<H, NSUB, D> sm;
    const int64_t b = blockIdx.x;
    const int sh = shot_of[b];
    StepArgs<float> a = shots[sh];
    const int64_t local = b - tile0[sh];
    const int64_t nstrip = a.ntx * (((a.L.nz + 7) / 8 + NSUB - 1) / NSUB);
    if (local >= nstrip) return;   // uniform per block
    const int64_t tot = a.L.total;
    a.p = a.buf0 + (int64_t)(j + 1) * tot;
    a.pm = a.buf0 + (int64_t)j * tot;
    a.out = a.buf0 + (int64_t)(j + 2) * tot;
    a.step = n;
    leap2d_strip<H, NSUB, D>(a, local % a.ntx, local / a.ntx, sm);
}

// Per-shot field copies between wavefield buffers, checkpoints and segment buffers
template <typename T>
struct ShotCopy {
    const T* a;           // batched forward: the shot's buf0 (steps n even: p^n) ...
    const T* b;           // ... and buf1; adjoint restore: the checkpoint slot base
    T* dst;               // checkpoint base (forward) or segment buffer (restore)
    int64_t total;        // padded field size
};

// forward, before step n: checkpoint k = [p^n, p^{n-1}] of every shot
template <typename T>
__global__ void k_ckpt_batch(const ShotCopy<T>* __restrict__ items, int n, int k) {
    const ShotCopy<T> it = items[blockIdx.y];
    const T* cur = (n & 1) ? it.b : it.a;
    const T* prev = (n & 1) ? it.a : it.b;
    T* slot = it.dst + (int64_t)k * 2 * it.total;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < it.total; i += (int64_t)gridDim.x * blockDim.x) {
        slot[i] = cur[i];
        slot[it.total + i] = prev[i];
    }
}

// adjoint, start of segment k: segment slots 0, 1 = p^{c-1}, p^c from checkpoint k
template <typename T>
__global__ void k_seg_restore_batch(const ShotCopy<T>* __restrict__ items, int k) {
    const ShotCopy<T> it = items[blockIdx.y];
    const T* slot = it.a + (int64_t)k * 2 * it.total;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < it.total; i += (int64_t)gridDim.x * blockDim.x) {
        it.dst[i] = slot[it.total + i];
        it.dst[it.total + i] = slot[i];
    }
}

// receivers only (after the last step)
template <typename T>
__global__ void k_receivers(PointSet<T> rec, const T* p, T* traces, int nt, int col) {
    record_receivers(rec, p, traces, nt, col, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, launch_threads());
}

// 3D: (x, y) tile of 32 x 8 columns marching in z with a register queue of the
// 2H + 1 values of its own column; x/y neighbours from a shared-memory copy of
// the current plane with its halo.
template <typename T, int H>
__global__ void __launch_bounds__(256) k_leap3d(StepArgs<T> a, int zchunk, int64_t nty) {
    constexpr int TX = 32, TY = 8;
    __shared__ T tile[TY + 2 * H][TX + 2 * H];
    __shared__ T acc[TY * TX];
    __shared__ T sadd[TY * TX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, blk * 256 + tid, launch_threads());
    const Layout& L = a.L;
    const int64_t x0 = (int64_t)blockIdx.x * TX, y0 = (int64_t)blockIdx.y * TY;
    const int64_t x = x0 + tx, y = y0 + ty;
    const int64_t zb = (int64_t)blockIdx.z * zchunk;
    const int64_t ze = min(zb + zchunk, L.nz);
    const bool col_ok = x < L.nx + H && y < L.ny + H;
    const bool valid = x < L.nx && y < L.ny;
    T q[2 * H + 1];
#pragma unroll
    for (int k = 0; k <= 2 * H; ++k) q[k] = col_ok ? a.p[L.idx(x, y, zb - H + k)] : (T)0;
    const T wv = a.src.n ? a.wavelet[a.step] : (T)0;
    for (int64_t z = zb; z < ze; ++z) {
        for (int i = tid; i < (TY + 2 * H) * (TX + 2 * H); i += TX * TY) {
            int ly = i / (TX + 2 * H), lx = i - ly * (TX + 2 * H);
            int64_t gx = x0 + lx - H, gy = y0 + ly - H;
            T v = 0;
            if (gx < L.nx + H && gy < L.ny + H) v = a.p[L.idx(gx, gy, z)];
            tile[ly][lx] = v;
        }
        sadd[tid] = (T)0;
        __syncthreads();
        {
            // the grouping of the TMA kernel (see there): exact zero on constants
            const T c = q[H];
            const T c6 = mul_rn((T)6, c);
            T s = 0;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const T g = add_rn(add_rn(add_rn(tile[ty + H][tx + H + k], tile[ty + H][tx + H - k]),
                                          add_rn(tile[ty + H + k][tx + H], tile[ty + H - k][tx + H])),
                                   add_rn(q[H + k], q[H - k]));
                s = fma_(a.w2[k], sub_rn(g, c6), s);
            }
            acc[tid] = s;
        }
        const int64_t origin = L.idx(x0, y0, z);
        tile_sources<T, TX, TY>(a.src, wv, origin, L.px, sadd, tid);
        __syncthreads();
        if (a.op.ptr) add_entries(a.op, (z * nty + blockIdx.y) * a.op.ntx + blockIdx.x, a.p, origin, acc, tid, 256);
        __syncthreads();
        if (valid) {
            int64_t qi = L.idx(x, y, z);
            T c = q[H];
            const T pmq = a.pm[qi];
            T u = c + ((c - pmq) + a.Kh[qi] * acc[tid]) + sadd[tid];
            if (a.dw && damp_box(L, a.dw, x, x, y, y, z)) u -= damp_g<T>(L, a.dw, a.da, x, y, z) * (u - pmq);
            a.out[qi] = u;
        }
#pragma unroll
        for (int k = 0; k < 2 * H; ++k) q[k] = q[k + 1];
        // plane z + 1 + H exists only while z + 1 < ze (the last allocated plane is nz + H - 1)
        q[2 * H] = (col_ok && z + 1 < ze) ? a.p[L.idx(x, y, z + 1 + H)] : (T)0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 3D leapfrog, FP32, with the plane tiles staged by TMA.  Each block marches a
// 32 x 8 column tile through its z chunk.  Plane z (with an x halo of 4 -- the
// 16-byte alignment of the box -- and a y halo of H) is fetched by one
// cp.async.bulk.tensor into a ring of NS shared-memory slots, NS - H - 1 planes
// ahead of use, each slot tracked by an mbarrier.  The z neighbours come from a
// register queue fed by the centre of plane z + H.  Every wait is bounded: on
// timeout the block records an error and leaves.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait; returns false once about one second has passed (or after 2^22
// polls, should the global timer not advance)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) break;
    }
    return false;
}

// Self-test of the bounded wait: one thread arms an mbarrier for bytes that no
// copy will ever deliver and waits with the same bound as the TMA kernels; the
// wait gives up and the kernel reports it through the error word.
__global__ void k_wait_selftest(int* err) {
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, 16);
    if (!mbar_wait_bounded(&bar, 0)) atomicExch(err, 1);
}

// compact corrections of the 3D tile planes (TileBins compact form): entries of
// tile plane t are [ptr[t], ptr[t + 1]), each an output slot (one byte), a 16-bit
// footprint code and an FP32 weight
struct Rows3 {
    const int32_t* ptr;
    const uint8_t* slot;
    const uint16_t* code;
    const float* w;
};

// Entries [e0, e1) of a tile plane: each warp takes chunks of 32 consecutive
// entries, four chunks at a time (four independent gathers in flight per
// thread); entries of one row are contiguous, so a segmented warp sum leaves one
// shared-memory atomic per row segment.  Values are read from p^n (L2).
__device__ __forceinline__ void add_entries3(const Rows3& r, int32_t e0, int32_t e1, const float* prow0,
                                             int64_t px, int64_t plane, float* acc, int tid) {
    constexpr int U = 4;
    const int lane = tid & 31;
    const int32_t warp_base = (tid & ~31) * U;
    for (int32_t base = e0 + warp_base; base < e1; base += 256 * U) {
        int32_t loc[U];
        float val[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t e = base + u * 32 + lane;
            ok[u] = e < e1;
            float v = 0.f;
            loc[u] = -1 - lane;
            if (ok[u]) {
                const int sl = r.slot[e];
                const int c = r.code[e];
                const int dx = (c & 31) - 16, dy = ((c >> 5) & 31) - 16, dz = (c >> 10) - 16;
                loc[u] = sl;
                v = r.w[e] * prow0[(int64_t)dz * plane + ((sl >> 5) + dy) * px + (sl & 31) + dx];
            }
            val[u] = v;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) seg_add(acc, loc[u], val[u], ok[u], lane);
    }
}

template <int H, int D>
struct Tma3D {
    static constexpr int TX = 32, TY = 8;
    static constexpr int BW = TX + 8;         // x halo 4 on each side (16-byte aligned box)
    static constexpr int BH = TY + 2 * H;
    static constexpr int NS = H + 1 + D;      // ring slots: planes z .. z + H + D (D planes in flight)
    static constexpr int PF = BW * BH;        // p plane with halo (floats)
    static constexpr int TF = TX * TY;        // p_prev or K tile (floats)
    static constexpr int SLOT = (PF + 2 * TF + 31) / 32 * 32;   // slot stride in floats (128-byte multiple)
    static constexpr uint32_t BYTES = (PF + 2 * TF) * 4;
};

// Laplacian (difference form) at the centre r0 of a staged plane, z neighbours from
// the register queue q (centre q[H + O]): sum_k w_k (((a + b) + (d + e)) + (f + g)
// - 6 c) over the six neighbours at distance k.  For a constant field each group
// is exactly zero in floating point (6 c rounds like the sum of the pairs), so the
// discrete operator annihilates constants.
template <int H, int O>
__device__ __forceinline__ float lap3_tma(const float* r0, const float (&q)[2 * H + 2], const float* w2) {
    constexpr int BW = 40;
    const float c = q[H + O];
    const float c6 = __fmul_rn(6.f, c);
    float sum = 0.f;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        const float g = __fadd_rn(__fadd_rn(__fadd_rn(r0[k], r0[-k]), __fadd_rn(r0[k * BW], r0[-k * BW])),
                                  __fadd_rn(q[H + O + k], q[H + O - k]));
        sum = fmaf(w2[k], __fsub_rn(g, c6), sum);
    }
    return sum;
}

// Each block marches a 32 x 8 column tile through its z chunk, two planes per
// iteration.  Ring slot k holds plane z (with an x halo of 4 and a y halo of H) of
// p^n, and the tiles of p^{n-1} and of K = dt^2 c^2 / h^2 at plane z: three
// cp.async.bulk.tensor copies on one mbarrier, issued when the slot's previous
// plane is done.  The z neighbours come from a register queue fed by the centres of
// planes z + H and z + H + 1.  The corrections of each tile plane are gathered by
// all threads (add_entries3): per entry a one-byte output slot, a 16-bit footprint
// code and an FP32 weight (7 bytes), the value read from p^n in global memory
// (L2).  Every wait is bounded: on timeout the block records an error, waits
// (bounded) for the planes already requested, and leaves.
template <int H, int D>
__global__ void __launch_bounds__(256, D <= 2 ? 6 : 5) k_leap3d_tma(StepArgs<float> a, const __grid_constant__ CUtensorMap tm,
                                                    const __grid_constant__ CUtensorMap tmm,
                                                    const __grid_constant__ CUtensorMap tmk, Rows3 rw, int zchunk,
                                                    int64_t nty, int* err) {
    using C = Tma3D<H, D>;
    constexpr int TX = C::TX, TY = C::TY, BW = C::BW, NS = C::NS, SLOT = C::SLOT, PF = C::PF, TF = C::TF;
    static_assert(NS >= H + 2, "planes z .. z + H + 1 are resident together");
    static_assert(BW == 40, "lap3_tma reads rows of 40 floats");
    extern __shared__ __align__(128) float dsm[];
    float* ring = dsm;                                  // NS * SLOT
    float* acc = ring + NS * SLOT;                      // [2][TY * TX]
    float* sadd = acc + 2 * TY * TX;                    // [2][TY * TX]
    uint64_t* bar = (uint64_t*)(sadd + 2 * TY * TX);    // NS
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, blk * 256 + tid, launch_threads());
    const Layout& L = a.L;
    const int64_t x0 = (int64_t)blockIdx.x * TX, y0 = (int64_t)blockIdx.y * TY;
    const int64_t x = x0 + tx, y = y0 + ty;
    const int64_t zb = (int64_t)blockIdx.z * zchunk;
    const int64_t ze = min(zb + zchunk, L.nz);
    const int64_t zlast = ze - 1 + H;                 // last p plane fetched
    const bool col_ok = x < L.nx + H && y < L.ny + H;
    const bool valid = x < L.nx && y < L.ny;
    const bool damped_xy = damp_box(L, a.dw, x0, x0 + TX - 1, y0, y0 + TY - 1, 0);
    // tensor rows: p plane z, tile row y0 - H at (H + 1 + z) py + y0; tile row y0 at + H
    auto prow = [&](int64_t z) { return (int)((H + 1 + z) * L.py + y0); };
    // slot for plane zz: p box always; the p_prev / K tiles only for planes the block updates
    auto issue = [&](int slot, int64_t zz) {
        const bool upd = zz < ze;
        mbar_expect_tx(&bar[slot], (uint32_t)(PF * 4 + (upd ? 2 * TF * 4 : 0)));
        float* dst = ring + slot * SLOT;
        tma_load_2d(dst, &tm, (int)(x0 - 4), prow(zz), &bar[slot]);
        if (upd) {
            tma_load_2d(dst + PF, &tmm, (int)x0, prow(zz) + H, &bar[slot]);
            tma_load_2d(dst + PF + TF, &tmk, (int)x0, prow(zz) + H, &bar[slot]);
        }
    };
    // bounded wait for plane zz of this chunk
    auto wait_plane = [&](int64_t zz) {
        const int ip = (int)(zz - zb);
        return mbar_wait_bounded(&bar[ip % NS], (uint32_t)((ip / NS) & 1));
    };
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < NS && zb + i <= zlast; ++i) issue(i, zb + i);
    float q[2 * H + 2];
#pragma unroll
    for (int k = 0; k < 2 * H; ++k) q[k] = col_ok ? a.p[L.idx(x, y, zb - H + k)] : 0.f;
    const float wv = a.src.n ? a.wavelet[a.step] : 0.f;
    const int64_t tile_z = nty * a.op.ntx;              // tiles per plane
    const int64_t tile0 = (int64_t)blockIdx.y * a.op.ntx + blockIdx.x;
    const bool src_me = tid < 8 * a.src.n;
    const int64_t s_idx = src_me ? a.src.idx[tid] : 0;
    const float s_w = src_me ? a.src.w[tid] : 0.f;
    int64_t qi = L.idx(x, y, zb);
    for (int64_t z = zb; z < ze; z += 2) {
        const bool two = z + 1 < ze;
        const int ia = (int)(z - zb);
        // entry ranges of the two tile planes (read while the planes are waited for)
        int32_t ea0 = 0, ea1 = 0, eb0 = 0, eb1 = 0;
        if (rw.ptr) {
            const int32_t* pp = rw.ptr + z * tile_z + tile0;
            ea0 = pp[0];
            ea1 = pp[1];
            if (two) {
                eb0 = pp[tile_z];
                eb1 = pp[tile_z + 1];
            }
        }
        bool ok = wait_plane(z) && wait_plane(z + H);
        if (two) ok = ok && wait_plane(z + 1) && wait_plane(z + 1 + H);
        // (after a failed wait the reads below see stale shared memory; the barrier
        // that follows them tells every thread, and the block leaves)
        const float* ra = ring + (ia % NS) * SLOT;           // plane z, row j <-> y0 - H + j
        const float* rb = ring + ((ia + 1) % NS) * SLOT;     // plane z + 1
        const int ci = (H + ty) * BW + 4 + tx;
        q[2 * H] = ring[((ia + H) % NS) * SLOT + ci];
        q[2 * H + 1] = two ? ring[((ia + H + 1) % NS) * SLOT + ci] : 0.f;
        const float pma = ra[PF + tid], kha = ra[PF + TF + tid];
        const float pmb = rb[PF + tid], khb = rb[PF + TF + tid];
        acc[tid] = lap3_tma<H, 0>(ra + ci, q, a.w2);
        acc[TX * TY + tid] = lap3_tma<H, 1>(rb + ci, q, a.w2);
        sadd[tid] = 0.f;
        sadd[TX * TY + tid] = 0.f;
        const int64_t origin = L.idx(x0, y0, z);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, 1);
                // issue nothing more, and wait (bounded) for every plane already issued
                // (planes z .. z + NS - 1), so that no copy is still landing in this
                // block's shared memory when it leaves
                const int64_t ziss = min(z + NS - 1, zlast);
                for (int64_t zp = z; zp <= ziss; ++zp) wait_plane(zp);
            }
            return;
        }
        if (src_me && s_w != 0.f) {
            const int64_t rel = s_idx - origin;
            if (rel >= 0) {
                const int64_t lz = rel / L.plane, r2 = rel - lz * L.plane;
                const int64_t ly = r2 / L.px, lx = r2 - ly * L.px;
                if (lz < (two ? 2 : 1) && ly < TY && lx < TX) atomicAdd(&sadd[lz * TX * TY + ly * TX + lx], s_w * wv);
            }
        }
        if (ea1 > ea0) add_entries3(rw, ea0, ea1, a.p + origin, L.px, L.plane, acc, tid);
        if (eb1 > eb0) add_entries3(rw, eb0, eb1, a.p + origin + L.plane, L.px, L.plane, acc + TX * TY, tid);
        __syncthreads();
        // the two slots are free (p_prev and K read above, the stencils done): the
        // planes NS further into them
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (z + NS <= zlast) issue(ia % NS, z + NS);
            if (two && z + 1 + NS <= zlast) issue((ia + 1) % NS, z + 1 + NS);
        }
        if (valid) {
            float u = q[H] + ((q[H] - pma) + kha * acc[tid]) + sadd[tid];
            if (damped_xy || (a.dw && z > L.nz - 1 - a.dw)) u -= damp_g<float>(L, a.dw, a.da, x, y, z) * (u - pma);
            a.out[qi] = u;
            if (two) {
                float ub = q[H + 1] + ((q[H + 1] - pmb) + khb * acc[TX * TY + tid]) + sadd[TX * TY + tid];
                if (damped_xy || (a.dw && z + 1 > L.nz - 1 - a.dw))
                    ub -= damp_g<float>(L, a.dw, a.da, x, y, z + 1) * (ub - pmb);
                a.out[qi + L.plane] = ub;
            }
        }
        qi += 2 * L.plane;
#pragma unroll
        for (int k = 0; k < 2 * H; ++k) q[k] = q[k + 2];
    }
    // planes fetched past the chunk that no iteration waited for (chunks shorter than H):
    // complete them before the block leaves
    bool ok = true;
    for (int64_t zz = ze; zz <= zlast; ++zz) ok = ok && wait_plane(zz);
    if (!ok && tid == 0) atomicExch(err, 1);
}

// Corrections of the modified Laplacian for a 3D step whose kernel applied the
// standard stencil only, over all IB rows of the grid at once:
//   out[q] += (1 - g(q)) K[q] sum_j w_j p[q + off_j]
// (g the absorbing-layer factor of the step, 0 outside the layer), entries as a
// 16-bit footprint code and an FP32 weight in row order.  A group of 8 lanes takes
// one row (a warp four rows), each lane up to U entries per round with their
// gathers in flight together, and the sum is added with a reduction that returns
// nothing (rows are distinct nodes), so no lane waits on it.
template <int U>
__global__ void __launch_bounds__(256) k_ib_add3(int64_t nrows, const int64_t* __restrict__ row_pad,
                                                 const int64_t* __restrict__ row_ptr,
                                                 const uint16_t* __restrict__ code, const float* __restrict__ w,
                                                 const float* __restrict__ p, const float* __restrict__ Kh,
                                                 float* out, Layout L, int dw, float da) {
    const int lane = threadIdx.x & 31, gl = lane & 7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto gather = [&](int64_t q, int c) {
        return p[q + (int64_t)((c >> 10) - 16) * L.plane + (int64_t)(((c >> 5) & 31) - 16) * L.px + ((c & 31) - 16)];
    };
    for (int64_t rb = warp * 4; rb < nrows; rb += nwarp * 4) {
        const int64_t r = rb + (lane >> 3);
        const bool act = r < nrows;
        const int64_t q = act ? row_pad[r] : 0;
        const int64_t j0 = act ? row_ptr[r] : 0, j1 = act ? row_ptr[r + 1] : 0;
        float v = 0.f;
        for (int64_t j = j0 + gl; j < j1; j += 8 * U) {
            float wv[U], pv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = j + 8 * u;
                const bool ok = e < j1;
                const int c = ok ? code[e] : 16 | (16 << 5) | (16 << 10);
                wv[u] = ok ? w[e] : 0.f;
                pv[u] = gather(q, c);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) v += wv[u] * pv[u];
        }
        v += __shfl_xor_sync(0xffffffffu, v, 4, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 2, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 1, 8);
        if (act && gl == 0) {
            float add = Kh[q] * v;
            if (dw) {
                const int64_t rel = q - L.base, z = rel / L.plane, rem = rel - z * L.plane;
                const int64_t y = rem / L.px, x = rem - y * L.px;
                add *= 1.f - damp_g<float>(L, dw, da, x, y, z);
            }
            atomicAdd(&out[q], add);
        }
    }
}

template <int H, int D>
static size_t tma3d_smem() {
    using C = Tma3D<H, D>;
    return sizeof(float) * ((size_t)C::NS * C::SLOT + 4 * C::TX * C::TY) + sizeof(uint64_t) * C::NS;
}

// planes in flight per block: 3 by default (IB_RING=2 or 5 selects 2 or 5, for tuning)
template <int H>
static void launch_leap3d_tma(const StepArgs<float>& a, const CUtensorMap& tm, const CUtensorMap& tmm,
                              const CUtensorMap& tmk, const Rows3& rw, int zchunk, int64_t nty, int* err, dim3 grid,
                              cudaStream_t s) {
    static const int ring = [] {
        const char* e = getenv("IB_RING");
        const int r = e ? atoi(e) : 3;
        return r == 5 || r == 2 ? r : 3;
    }();
    const dim3 blk(32, 8);
    if (ring == 2) {
        k_leap3d_tma<H, 2><<<grid, blk, tma3d_smem<H, 2>(), s>>>(a, tm, tmm, tmk, rw, zchunk, nty, err);
    } else if (ring == 5) {
        const size_t sm = tma3d_smem<H, 5>();
        cudaFuncSetAttribute(k_leap3d_tma<H, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_leap3d_tma<H, 5><<<grid, blk, sm, s>>>(a, tm, tmm, tmk, rw, zchunk, nty, err);
    } else {
        k_leap3d_tma<H, 3><<<grid, blk, tma3d_smem<H, 3>(), s>>>(a, tm, tmm, tmk, rw, zchunk, nty, err);
    }
}

// ---------------------------------------------------------------------------
// 3D step on x-pairs: the 64 x 8 column tile of a block is marched in z two
// planes per iteration like k_leap3d_tma, with each thread computing two
// x-adjacent points.  The x and y neighbours of the pair come in as 8-byte
// shared-memory loads (the x row -4 .. +5 in five, each y neighbour pair in one)
// and the waits, barriers and address arithmetic of an iteration are shared by
// four points instead of two.  The corrections are added by k_ib_add3 after the
// launch; sources touch shared memory only in the blocks that hold one.
// ---------------------------------------------------------------------------
template <int H, int D>
struct Tma3P {
    static constexpr int TX = 64, TY = 8;
    static constexpr int BW = TX + 8;         // x halo 4 on each side (16-byte aligned box)
    static constexpr int BH = TY + 2 * H;
    static constexpr int NS = H + 1 + D;      // ring slots: planes z .. z + H + D
    static constexpr int PF = (BW * BH + 31) / 32 * 32;   // p plane, padded to 128 bytes
    static constexpr int TF = TX * TY;
    static constexpr int SLOT = PF + 2 * TF;
};

// Laplacians of the pair centred at r0[0], r0[1] (r0 8-byte aligned, rows of 72
// floats), z neighbours from the register queue q (centre q[H + O]); the grouping
// and rounding of lap3_tma for each point
template <int H, int O>
__device__ __forceinline__ float2 lap3_pair(const float* r0, const float2 (&q)[2 * H + 2], const float* w2) {
    constexpr int BW = 72;
    float2 xv[5];   // r0[-4 .. 5]
#pragma unroll
    for (int j = 0; j < 5; ++j) xv[j] = *reinterpret_cast<const float2*>(r0 + 2 * j - 4);
    auto X = [&](int o) -> float {
        const int j = o + 4;
        return (j & 1) ? xv[j >> 1].y : xv[j >> 1].x;
    };
    const float2 c = q[H + O];
    const float c6a = __fmul_rn(6.f, c.x), c6b = __fmul_rn(6.f, c.y);
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        const float2 yp = *reinterpret_cast<const float2*>(r0 + k * BW);
        const float2 ym = *reinterpret_cast<const float2*>(r0 - k * BW);
        const float ga = __fadd_rn(__fadd_rn(__fadd_rn(X(k), X(-k)), __fadd_rn(yp.x, ym.x)),
                                   __fadd_rn(q[H + O + k].x, q[H + O - k].x));
        const float gb = __fadd_rn(__fadd_rn(__fadd_rn(X(1 + k), X(1 - k)), __fadd_rn(yp.y, ym.y)),
                                   __fadd_rn(q[H + O + k].y, q[H + O - k].y));
        sa = fmaf(w2[k], __fsub_rn(ga, c6a), sa);
        sb = fmaf(w2[k], __fsub_rn(gb, c6b), sb);
    }
    return make_float2(sa, sb);
}

template <int H, int D>
__global__ void __launch_bounds__(256, 3) k_leap3d_tma2(StepArgs<float> a, const __grid_constant__ CUtensorMap tm,
                                                        const __grid_constant__ CUtensorMap tmm,
                                                        const __grid_constant__ CUtensorMap tmk, int zchunk,
                                                        int* err) {
    using C = Tma3P<H, D>;
    constexpr int TX = C::TX, TY = C::TY, BW = C::BW, NS = C::NS, SLOT = C::SLOT, PF = C::PF, TF = C::TF;
    static_assert(NS >= H + 2, "planes z .. z + H + 1 are resident together");
    static_assert(BW == 72 && H <= 4, "lap3_pair reads rows of 72 floats, x halo 4");
    extern __shared__ __align__(128) float dsm[];
    float* ring = dsm;                                  // NS * SLOT
    float* sadd = ring + NS * SLOT;                     // [2][TY * TX]
    uint64_t* bar = (uint64_t*)(sadd + 2 * TY * TX);    // NS
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step, blk * 256 + tid, launch_threads());
    const Layout& L = a.L;
    const int64_t x0 = (int64_t)blockIdx.x * TX, y0 = (int64_t)blockIdx.y * TY;
    const int64_t xa = x0 + 2 * tx, y = y0 + ty;        // this thread's points: (xa, y), (xa + 1, y)
    const int64_t zb = (int64_t)blockIdx.z * zchunk;
    const int64_t ze = min(zb + zchunk, L.nz);
    const int64_t zlast = ze - 1 + H;
    const bool va = xa < L.nx && y < L.ny, vb = xa + 1 < L.nx && y < L.ny;
    const bool damped_xy = damp_box(L, a.dw, x0, x0 + TX - 1, y0, y0 + TY - 1, 0);
    auto prow = [&](int64_t z) { return (int)((H + 1 + z) * L.py + y0); };
    auto issue = [&](int slot, int64_t zz) {
        const bool upd = zz < ze;
        mbar_expect_tx(&bar[slot], (uint32_t)(BW * C::BH * 4 + (upd ? 2 * TF * 4 : 0)));
        float* dst = ring + slot * SLOT;
        tma_load_2d(dst, &tm, (int)(x0 - 4), prow(zz), &bar[slot]);
        if (upd) {
            tma_load_2d(dst + PF, &tmm, (int)x0, prow(zz) + H, &bar[slot]);
            tma_load_2d(dst + PF + TF, &tmk, (int)x0, prow(zz) + H, &bar[slot]);
        }
    };
    auto wait_plane = [&](int64_t zz) {
        const int ip = (int)(zz - zb);
        return mbar_wait_bounded(&bar[ip % NS], (uint32_t)((ip / NS) & 1));
    };
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // does a source corner fall in this block's columns and z chunk? (block-uniform)
    int src_here = 0;
    const float wv = a.src.n ? a.wavelet[a.step] : 0.f;
    const bool src_me = tid < 8 * a.src.n;
    int64_t s_rel = -1;   // this thread's corner, relative to node (x0, y0, zb)
    float s_val = 0.f;
    if (src_me && a.src.w[tid] != 0.f) {
        const int64_t rel = a.src.idx[tid] - L.idx(x0, y0, zb);
        if (rel >= 0) {
            const int64_t lz = rel / L.plane, r2 = rel - lz * L.plane;
            const int64_t ly = r2 / L.px, lx = r2 - ly * L.px;
            if (lz < ze - zb && ly < TY && lx < TX) {
                s_rel = rel;
                s_val = a.src.w[tid] * wv;
            }
        }
    }
    src_here = __syncthreads_or(s_rel >= 0);
    if (tid == 0)
        for (int i = 0; i < NS && zb + i <= zlast; ++i) issue(i, zb + i);
    float2 q[2 * H + 2];
    {
        const bool ca = xa < L.nx + H && y < L.ny + H, cb = xa + 1 < L.nx + H && y < L.ny + H;
#pragma unroll
        for (int k = 0; k < 2 * H; ++k) {
            const int64_t i = L.idx(xa, y, zb - H + k);
            q[k] = make_float2(ca ? a.p[i] : 0.f, cb ? a.p[i + 1] : 0.f);
        }
    }
    int64_t qi = L.idx(xa, y, zb);
    const int ci = (H + ty) * BW + 4 + 2 * tx;   // pair centre in a slot's p plane
    const int ti = ty * TX + 2 * tx;             // pair in a slot's p_prev / K tile
    for (int64_t z = zb; z < ze; z += 2) {
        const bool two = z + 1 < ze;
        const int ia = (int)(z - zb);
        bool ok = wait_plane(z) && wait_plane(z + H);
        if (two) ok = ok && wait_plane(z + 1) && wait_plane(z + 1 + H);
        // (after a failed wait the reads below see stale shared memory; the barrier
        // that follows them tells every thread, and the block leaves)
        const float* ra = ring + (ia % NS) * SLOT;
        const float* rb = ring + ((ia + 1) % NS) * SLOT;
        q[2 * H] = *reinterpret_cast<const float2*>(ring + ((ia + H) % NS) * SLOT + ci);
        q[2 * H + 1] = two ? *reinterpret_cast<const float2*>(ring + ((ia + H + 1) % NS) * SLOT + ci)
                           : make_float2(0.f, 0.f);
        const float2 pma = *reinterpret_cast<const float2*>(ra + PF + ti);
        const float2 kha = *reinterpret_cast<const float2*>(ra + PF + TF + ti);
        const float2 pmb = *reinterpret_cast<const float2*>(rb + PF + ti);
        const float2 khb = *reinterpret_cast<const float2*>(rb + PF + TF + ti);
        const float2 la = lap3_pair<H, 0>(ra + ci, q, a.w2);
        const float2 lb = lap3_pair<H, 1>(rb + ci, q, a.w2);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, 1);
                const int64_t ziss = min(z + NS - 1, zlast);
                for (int64_t zp = z; zp <= ziss; ++zp) wait_plane(zp);
            }
            return;
        }
        // the two slots are free: the planes NS further into them
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (z + NS <= zlast) issue(ia % NS, z + NS);
            if (two && z + 1 + NS <= zlast) issue((ia + 1) % NS, z + 1 + NS);
        }
        float2 ua, ub;
        ua.x = q[H].x + ((q[H].x - pma.x) + kha.x * la.x);
        ua.y = q[H].y + ((q[H].y - pma.y) + kha.y * la.y);
        ub.x = q[H + 1].x + ((q[H + 1].x - pmb.x) + khb.x * lb.x);
        ub.y = q[H + 1].y + ((q[H + 1].y - pmb.y) + khb.y * lb.y);
        if (src_here) {   // block-uniform
            float2* s2 = reinterpret_cast<float2*>(sadd);
            s2[tid] = make_float2(0.f, 0.f);
            s2[TX * TY / 2 + tid] = make_float2(0.f, 0.f);
            __syncthreads();
            if (s_rel >= 0) {
                const int64_t r = s_rel - (z - zb) * L.plane;
                if (r >= 0) {
                    const int64_t lz = r / L.plane, r2 = r - lz * L.plane;
                    const int64_t ly = r2 / L.px, lx = r2 - ly * L.px;
                    if (lz < (two ? 2 : 1)) atomicAdd(&sadd[lz * TX * TY + ly * TX + lx], s_val);
                }
            }
            __syncthreads();
            const float2 sa = s2[ti / 2], sb = s2[TX * TY / 2 + ti / 2];
            ua.x += sa.x;
            ua.y += sa.y;
            ub.x += sb.x;
            ub.y += sb.y;
        }
        if (damped_xy || (a.dw && z + 1 > L.nz - 1 - a.dw)) {
            ua.x -= damp_g<float>(L, a.dw, a.da, xa, y, z) * (ua.x - pma.x);
            ua.y -= damp_g<float>(L, a.dw, a.da, xa + 1, y, z) * (ua.y - pma.y);
            if (two) {
                ub.x -= damp_g<float>(L, a.dw, a.da, xa, y, z + 1) * (ub.x - pmb.x);
                ub.y -= damp_g<float>(L, a.dw, a.da, xa + 1, y, z + 1) * (ub.y - pmb.y);
            }
        }
        if (va && vb) {
            *reinterpret_cast<float2*>(a.out + qi) = ua;
            if (two) *reinterpret_cast<float2*>(a.out + qi + L.plane) = ub;
        } else if (va) {
            a.out[qi] = ua.x;
            if (two) a.out[qi + L.plane] = ub.x;
        }
        qi += 2 * L.plane;
#pragma unroll
        for (int k = 0; k < 2 * H; ++k) q[k] = q[k + 2];
    }
    bool ok = true;
    for (int64_t zz = ze; zz <= zlast; ++zz) ok = ok && wait_plane(zz);
    if (!ok && tid == 0) atomicExch(err, 1);
}

template <int H, int D>
static size_t tma3p_smem() {
    using C = Tma3P<H, D>;
    return sizeof(float) * ((size_t)C::NS * C::SLOT + 2 * C::TX * C::TY) + sizeof(uint64_t) * C::NS;
}

// x-pair kernel: 3 planes in flight beyond the ones read (IB_RING=2: 2).  At
// 512^2 x 384, order 8: 325 us per launch with 3, 383 us with 2 (three blocks of
// 74 KB or 65 KB per SM either way).
template <int H>
static void launch_leap3d_tma2(const StepArgs<float>& a, const CUtensorMap& tm, const CUtensorMap& tmm,
                               const CUtensorMap& tmk, int zchunk, int* err, dim3 grid, cudaStream_t s) {
    static const int ring = [] {
        const char* e = getenv("IB_RING");
        return e && atoi(e) == 2 ? 2 : 3;
    }();
    const dim3 blk(32, 8);
    if (ring == 3) {
        static const size_t sm = tma3p_smem<H, 3>();
        static const bool attr = (cudaFuncSetAttribute(k_leap3d_tma2<H, 3>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                                  true);
        (void)attr;
        k_leap3d_tma2<H, 3><<<grid, blk, sm, s>>>(a, tm, tmm, tmk, zchunk, err);
    } else {
        static const size_t sm = tma3p_smem<H, 2>();
        static const bool attr = (cudaFuncSetAttribute(k_leap3d_tma2<H, 2>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                                  true);
        (void)attr;
        k_leap3d_tma2<H, 2><<<grid, blk, sm, s>>>(a, tm, tmm, tmk, zchunk, err);
    }
}

// ---------------------------------------------------------------------------
// 2D staggered pressure-velocity
//   v_a[j] (at j + e_a/2) += bh_a[j] (sum_k c_k (p[j + k e_a] - p[j - (k-1) e_a]) + IB)
//   p[j] += kh[j] (sum_a sum_k c_k (v_a[j + (k-1) e_a] - v_a[j - k e_a]) + IB) + src
// with bh_a = dt / (rho h) and kh = dt rho c^2 / h
// ---------------------------------------------------------------------------
// Producer-side partial sums of the staggered corrections.  A correction row
// sum_e w_e f[col_e] is split by the step tile that holds col_e: the kernel
// that has just produced f on that tile forms partial[pid] = the sum over the
// row's entries there (values read from shared memory), and the kernel that
// consumes the row adds its partials (1-4 per row) while it loads its tile.
// No kernel gathers correction columns from global memory.
template <typename T>
struct StagPlan {
    // producer side (this kernel writes `out`): per tile, pid positions
    // [qptr[t], qptr[t+1]) and entries [eptr[t], eptr[t+1])
    const int32_t* qptr;
    const int32_t* qpid;     // global pid of each position
    const int32_t* eptr;
    const int32_t* emeta;    // field << 31 | (pid position - qptr[t]) << 11 | slot (lz * TX + lx) of the column
    const T* ew;
    T* out;
    int max_q;               // largest pid count of a tile
    // consumer side (this kernel reads `in`): per tile, rows [rptr[t], rptr[t+1])
    const int32_t* rptr;
    const int32_t* rslot;    // target << 24 | slot of the row node
    const int32_t* rpb;      // pid range of the row
    const int32_t* rpe;
    const T* in;
    int64_t n_in;            // partial sums in `in`
};

template <typename T>
struct StagArgs {
    Layout L;
    StagPlan<T> pv;          // v kernel: consumes partials of p, produces those of v
    StagPlan<T> pp;          // p kernel: consumes partials of v, produces those of p
    const uint8_t* src_tile; // per step tile: a source corner lies in it
    const int* step_base;    // device step offset added to step / rec_step (graph replays)
    T c1[4];             // staggered weights for offsets +1/2 .. +(M-1)/2
    T* p;
    T* vx;
    T* vz;
    const T* bx;
    const T* bz;
    const T* kp;
    TileView<T> gx, gz, dx, dz;
    PointSet<T> src;     // weights include dt / h^d
    const T* wavelet;
    int step;
    PointSet<T> rec;
    T* traces;
    int nt;
    int rec_step;
};

// consumer side: correction of row i of this tile's list = sum of its partials
template <typename T>
__device__ __forceinline__ T plan_row_sum(const StagPlan<T>& P, int32_t i) {
    T c = 0;
    for (int32_t q = P.rpb[i]; q < P.rpe[i]; ++q) c += P.in[q];
    return c;
}

// producer side, first part: stage up to STG of this tile's entries in shared memory
template <typename T, int STG>
__device__ __forceinline__ int32_t plan_stage(const StagPlan<T>& P, int64_t tile, int32_t* smeta, T* sw, int tid) {
    const int32_t e0 = P.eptr[tile], e1 = P.eptr[tile + 1];
    const int32_t n = e1 - e0 < STG ? e1 - e0 : STG;
    for (int32_t i = tid; i < n; i += 256) {
        cp_async<4>(&smeta[i], P.emeta + e0 + i, true);
        cp_async<(int)sizeof(T)>(&sw[i], P.ew + e0 + i, true);
    }
    return n;
}

// producer side: partial[pid] = sum of w * fnew[field][slot] over the pid's entries in this tile.
// A tile's entries are ordered by their rank within the pid, then by pid, so
// the lanes of a warp add into different partial sums.  The first `nst`
// entries were staged in shared memory while the tile loaded.
template <typename T, int SLOTS>
__device__ __forceinline__ void plan_produce(const StagPlan<T>& P, int64_t tile, const T* fnew, T* psum,
                                             const int32_t* smeta, const T* sw, int32_t nst, int tid) {
    const int32_t q0 = P.qptr[tile], nq = P.qptr[tile + 1] - q0;
    const int32_t e0 = P.eptr[tile], e1 = P.eptr[tile + 1];
    for (int32_t k = tid; k < nq; k += 256) psum[k] = (T)0;
    __syncthreads();
    for (int32_t i = tid; i < nst; i += 256) {
        const uint32_t mm = (uint32_t)smeta[i];
        atomicAdd(&psum[(mm >> 11) & 0xfffff], sw[i] * fnew[(mm >> 31) * SLOTS + (mm & 0x7ff)]);
    }
    constexpr int U = 8;
    for (int32_t base = e0 + nst + tid; base < e1; base += 256 * U) {
        int32_t m[U];
        T w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t e = base + u * 256;
            m[u] = e < e1 ? P.emeta[e] : 0;
            w[u] = e < e1 ? P.ew[e] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (base + u * 256 >= e1) continue;
            const uint32_t mm = (uint32_t)m[u];
            atomicAdd(&psum[(mm >> 11) & 0xfffff], w[u] * fnew[(mm >> 31) * SLOTS + (mm & 0x7ff)]);
        }
    }
    __syncthreads();
    for (int32_t k = tid; k < nq; k += 256) P.out[P.qpid[q0 + k]] = psum[k];
}

// v^{n+1/2} = v^{n-1/2} + (dt / rho) G_mod p^n on a 64 x TZ tile (256 threads as 64 x 4,
// TZ / 4 points per thread); the p tile and the producer entries arrive by cp.async
template <typename T, int H, int TX, int TZ, int MAXQ, int STG>
__global__ void __launch_bounds__(256, 4) k_stag_v2d(StagArgs<T> a) {
    static_assert(TX == 64 && TZ % 4 == 0, "64-wide tiles, 4 thread rows");
    constexpr int NP = TZ / 4, SL = TZ * TX;
    __shared__ __align__(16) T tile[TZ + 2 * H][TX + 2 * H];
    __shared__ T acc[2 * SL];                        // a_x, a_z; then the new v_x, v_z
    __shared__ T psum[MAXQ];
    __shared__ int32_t smeta[STG];
    __shared__ T sw[STG];
    const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    const int64_t x0 = (int64_t)blockIdx.x * TX, z0 = (int64_t)blockIdx.y * TZ;
    const Layout& L = a.L;
    const int64_t origin = L.base + z0 * L.px + x0;
    {
        const T* pb = a.p + origin - H * L.px - H;
#pragma unroll
        for (int lz = ty; lz < TZ + 2 * H; lz += 4) {
            const bool zok = z0 + lz - H < L.nz + H;
            const T* row = pb + lz * L.px;
            for (int lx = tx; lx < TX + 2 * H; lx += 64) {
                const bool ok = zok && x0 + lx - H < L.nx + H;
                cp_async<(int)sizeof(T)>(&tile[lz][lx], ok ? row + lx : a.p, ok);
            }
        }
    }
    const int32_t nst = plan_stage<T, STG>(a.pv, blk, smeta, sw, tid);
    cp_async_commit();
    const int sb = a.step_base ? *a.step_base : 0;
    record_receivers(a.rec, a.p, a.traces, a.nt, sb + a.rec_step, blk * 256 + tid, launch_threads());
    const int32_t r0 = a.pv.rptr[blk], r1 = a.pv.rptr[blk + 1];
    // the update's own operands and this tile's row corrections while the copies fly
    T vx[NP], vz[NP], bx[NP], bz[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int lz = ty + 4 * k;
        const bool in = x0 + tx < L.nx && z0 + lz < L.nz;
        const int64_t q = origin + lz * L.px + tx;
        vx[k] = in ? a.vx[q] : (T)0;
        vz[k] = in ? a.vz[q] : (T)0;
        bx[k] = in ? a.bx[q] : (T)0;
        bz[k] = in ? a.bz[q] : (T)0;
    }
    T corr = 0;
    int32_t cslot = 0;
    if (r0 + tid < r1) {
        corr = plan_row_sum(a.pv, r0 + tid);
        cslot = a.pv.rslot[r0 + tid];
    }
    cp_async_wait_all();
    __syncthreads();
    T ax[NP], az[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int lz = ty + 4 * k;
        T sx = 0, sz = 0;
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            sx += a.c1[j - 1] * (tile[lz + H][tx + H + j] - tile[lz + H][tx + H - j + 1]);
            sz += a.c1[j - 1] * (tile[lz + H + j][tx + H] - tile[lz + H - j + 1][tx + H]);
        }
        ax[k] = sx;
        az[k] = sz;
    }
    if (r1 > r0) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            acc[(ty + 4 * k) * TX + tx] = ax[k];
            acc[SL + (ty + 4 * k) * TX + tx] = az[k];
        }
        __syncthreads();
        for (int32_t i = r0 + tid; i < r1; i += 256) {
            if (i >= r0 + 256) {
                corr = plan_row_sum(a.pv, i);
                cslot = a.pv.rslot[i];
            }
            atomicAdd(&acc[(cslot >> 24) * SL + (cslot & 0xffffff)], corr);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            ax[k] = acc[(ty + 4 * k) * TX + tx];
            az[k] = acc[SL + (ty + 4 * k) * TX + tx];
        }
    }
    const bool produce = a.pv.out != nullptr && a.pv.eptr[blk + 1] > a.pv.eptr[blk];
    if (produce) __syncthreads();     // acc is reused for the new values
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int lz = ty + 4 * k;
        const T nvx = vx[k] + bx[k] * ax[k];
        const T nvz = vz[k] + bz[k] * az[k];
        if (produce) {
            acc[lz * TX + tx] = nvx;
            acc[SL + lz * TX + tx] = nvz;
        }
        if (x0 + tx >= L.nx || z0 + lz >= L.nz) continue;
        const int64_t q = origin + lz * L.px + tx;
        a.vx[q] = nvx;
        a.vz[q] = nvz;
    }
    if (produce) plan_produce<T, SL>(a.pv, blk, acc, psum, smeta, sw, nst, tid);
}

// p^{n+1} = p^n + dt rho c^2 D_mod v^{n+1/2} (+ source) on a 64 x TZ tile
template <typename T, int H, int TX, int TZ, int MAXQ, int STG>
__global__ void __launch_bounds__(256, 4) k_stag_p2d(StagArgs<T> a) {
    static_assert(TX == 64 && TZ % 4 == 0, "64-wide tiles, 4 thread rows");
    constexpr int NP = TZ / 4, SL = TZ * TX;
    __shared__ __align__(16) T tvx[TZ][TX + 2 * H];
    __shared__ __align__(16) T tvz[TZ + 2 * H][TX];
    __shared__ T acc[SL];
    __shared__ T psum[MAXQ];
    __shared__ int32_t smeta[STG];
    __shared__ T sw[STG];
    const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    const int64_t x0 = (int64_t)blockIdx.x * TX, z0 = (int64_t)blockIdx.y * TZ;
    const Layout& L = a.L;
    const int64_t origin = L.base + z0 * L.px + x0;
    {
        const T* vb = a.vx + origin - H;
#pragma unroll
        for (int lz = ty; lz < TZ; lz += 4) {
            const bool zok = z0 + lz < L.nz + H;
            const T* row = vb + lz * L.px;
            for (int lx = tx; lx < TX + 2 * H; lx += 64) {
                const bool ok = zok && x0 + lx - H < L.nx + H;
                cp_async<(int)sizeof(T)>(&tvx[lz][lx], ok ? row + lx : a.vx, ok);
            }
        }
        const T* wb = a.vz + origin - H * L.px;
        const bool xok = x0 + tx < L.nx + H;
#pragma unroll
        for (int lz = ty; lz < TZ + 2 * H; lz += 4) {
            const bool ok = xok && z0 + lz - H < L.nz + H;
            cp_async<(int)sizeof(T)>(&tvz[lz][tx], ok ? wb + lz * L.px + tx : a.vz, ok);
        }
    }
    const int32_t nst = plan_stage<T, STG>(a.pp, blk, smeta, sw, tid);
    cp_async_commit();
    const int32_t r0 = a.pp.rptr[blk], r1 = a.pp.rptr[blk + 1];
    T pv[NP], kv[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int lz = ty + 4 * k;
        const bool in = x0 + tx < L.nx && z0 + lz < L.nz;
        const int64_t q = origin + lz * L.px + tx;
        pv[k] = in ? a.p[q] : (T)0;
        kv[k] = in ? a.kp[q] : (T)0;
    }
    T corr = 0;
    int32_t cslot = 0;
    if (r0 + tid < r1) {
        corr = plan_row_sum(a.pp, r0 + tid);
        cslot = a.pp.rslot[r0 + tid];
    }
    const bool has_src = a.src.n > 0 && a.src_tile[blk] != 0;
    if (has_src || r1 > r0)
        for (int i = tid; i < SL; i += 256) acc[i] = (T)0;
    cp_async_wait_all();
    __syncthreads();
    T s[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int lz = ty + 4 * k;
        T sum = 0;
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            sum += a.c1[j - 1] * (tvx[lz][tx + H + j - 1] - tvx[lz][tx + H - j]);
            sum += a.c1[j - 1] * (tvz[lz + H + j - 1][tx] - tvz[lz + H - j][tx]);
        }
        s[k] = pv[k] + kv[k] * sum;
    }
    if (has_src || r1 > r0) {
        // acc collects kp * corrections and the source term of this tile
        const T wv = has_src ? a.wavelet[(a.step_base ? *a.step_base : 0) + a.step] : (T)0;
        tile_sources<T, TX, TZ>(a.src, wv, origin, L.px, acc, tid);
        for (int32_t i = r0 + tid; i < r1; i += 256) {
            if (i >= r0 + 256) {
                corr = plan_row_sum(a.pp, i);
                cslot = a.pp.rslot[i];
            }
            const int sl = cslot & 0xffffff;
            atomicAdd(&acc[sl], a.kp[origin + (sl / TX) * L.px + (sl % TX)] * corr);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NP; ++k) s[k] += acc[(ty + 4 * k) * TX + tx];
    }
    const bool produce = a.pp.out != nullptr && a.pp.eptr[blk + 1] > a.pp.eptr[blk];
    if (produce) __syncthreads();
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int lz = ty + 4 * k;
        if (produce) acc[lz * TX + tx] = s[k];
        if (x0 + tx >= L.nx || z0 + lz >= L.nz) continue;
        a.p[origin + lz * L.px + tx] = s[k];
    }
    if (produce) plan_produce<T, SL>(a.pp, blk, acc, psum, smeta, sw, nst, tid);
}

// ---------------------------------------------------------------------------
// 2D adjoint of the leapfrog map and the velocity gradient
//   mu^m = 2 mu^{m+1} - mu^{m+2} + mask (L^T (K mu^{m+1})) + R^T res^{m-1}
//   g   += mu^m (2 / c) (p^m - 2 p^{m-1} + p^{m-2} - s^{m-1})
//   gw[m-1] = S . mu^m
// ---------------------------------------------------------------------------
template <typename T>
struct AdjArgs {
    Layout L;
    T w2[5];
    const T* mu;         // mu^{m+1}
    const T* mum;        // mu^{m+2}
    T* out;              // mu^m (may alias mum)
    const T* Kh;         // dt^2 c^2 / h^2
    const uint8_t* mask;
    T two_dt_over_h;     // 2 dt / h  (2 / c = two_dt_over_h / sqrt(Kh))
    TileView<T> opT;     // transposed corrections, keyed by column node
    RowView<T> inj;      // receiver injection: col = receiver id
    const T* res;        // [nrec][nt]
    int nt;
    int m;
    const T* pm0;        // p^m
    const T* pm1;        // p^{m-1}
    const T* pm2;        // p^{m-2}
    T* grad;             // padded accumulator
    PointSet<T> src;
    const T* wavelet;
    T* gw;               // [nt] or null
    int dw;              // absorbing layer (as StepArgs); the stored multiplier is
    T da;                // nu^m = mu^m / (1 + a)
};

// one adjoint tile (bx, bz); shared arrays from the calling kernel
template <typename T, int H, int TX, int TZ>
__device__ __forceinline__ void adj2d_tile(const AdjArgs<T>& a, int64_t bx, int64_t bz, T (*tile)[TX + 8], T* tmu,
                                           T* acc, T* sw) {
    static_assert((TZ * TX) % 256 == 0, "whole points per thread");
    constexpr int W = TX + 8, V = 16 / (int)sizeof(T), CHR = W / V;
    constexpr int PT = TZ * TX / 256, NT = (TZ + 2 * H) * W;
    static_assert(H <= 4 && TX % 64 == 0, "columns x0-4 .. x0+TX+3 in 16-byte chunks");
    const int tid = threadIdx.x;
    const int64_t x0 = bx * TX, z0 = bz * TZ;
    const Layout& L = a.L;
    const int64_t origin = L.base + z0 * L.px + x0;
    const int64_t tile_id = bz * a.opT.ntx + bx;
    // K and mu halo tiles arrive by 16-byte cp.async: rows z0-H .. z0+TZ+H-1, columns
    // x0-4 .. x0+TX+3 (x0-4 is 16-byte aligned: the row pitch is a multiple of 32
    // elements).  Rows past nz+H-1 and chunks that would end past the allocation are
    // zero-filled; columns past nx+H-1 feed no stored point ...
    for (int i = tid; i < (TZ + 2 * H) * CHR; i += 256) {
        const int r = i / CHR, c = i - r * CHR;
        const int64_t z = z0 - H + r;
        const int64_t q = (z + H + 1) * L.px + x0 - 4 + V * c;
        const bool ok = z < L.nz + H && q + V <= L.total;
        cp_async<16>(&tile[r][V * c], ok ? a.Kh + q : a.Kh, ok);
        cp_async<16>(&tmu[r * W + V * c], ok ? a.mu + q : a.mu, ok);
    }
    cp_async_commit();
    for (int i = tid; i < TZ * TX; i += 256) sw[i] = (T)0;
    // ... while this thread's operands and the tile's entry ranges load
    T mu_v[PT], mum_v[PT], kh_v[PT], p0_v[PT], p1_v[PT], p2_v[PT], g_v[PT];
    bool msk[PT];
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j, lz = i / TX, lx = i - lz * TX;
        const bool in = x0 + lx < L.nx && z0 + lz < L.nz;
        const int64_t q = origin + lz * L.px + lx;
        mu_v[j] = in ? a.mu[q] : (T)0;
        mum_v[j] = in ? a.mum[q] : (T)0;
        kh_v[j] = in ? a.Kh[q] : (T)0;
        msk[j] = in ? a.mask[q] != 0 : false;
        p0_v[j] = in ? a.pm0[q] : (T)0;
        p1_v[j] = in ? a.pm1[q] : (T)0;
        p2_v[j] = in ? a.pm2[q] : (T)0;
        g_v[j] = in ? a.grad[q] : (T)0;
    }
    int32_t e0 = 0, e1 = 0, j0 = 0, j1 = 0;
    if (a.opT.ptr) {
        e0 = a.opT.ptr[tile_id];
        e1 = a.opT.ptr[tile_id + 1];
    }
    if (a.inj.tile_ptr) {
        j0 = a.inj.tile_ptr[tile_id];
        j1 = a.inj.tile_ptr[tile_id + 1];
    }
    cp_async_wait_all();
    __syncthreads();
    for (int i = tid; i < NT; i += 256) (&tile[0][0])[i] *= tmu[i];
    __syncthreads();
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        T c = tile[lz + H][lx + 4];
        T s = 0;
#pragma unroll
        for (int k = 1; k <= H; ++k)
            s += a.w2[k] * (((tile[lz + H][lx + 4 + k] - c) + (tile[lz + H][lx + 4 - k] - c)) +
                            ((tile[lz + H + k][lx + 4] - c) + (tile[lz + H - k][lx + 4] - c)));
        acc[i] = s;
    }
    tile_sources<T, TX, TZ>(a.src, (T)1, origin, L.px, sw, tid);
    __syncthreads();
    for (int32_t e = e0 + tid; e < e1; e += 256) {
        int64_t s = origin + a.opT.src[e];
        atomicAdd(&acc[a.opT.loc[e]], a.opT.w[e] * (a.Kh[s] * a.mu[s]));
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j;
        if (!msk[j]) acc[i] = (T)0;
    }
    __syncthreads();
    if (j1 > j0) {
        const int warp = tid >> 5, lane = tid & 31;
        for (int k = j0 + warp; k < j1; k += 8) {
            const int32_t r = a.inj.perm[k];
            const int64_t q = a.inj.row_pad[r];
            T s = 0;
            for (int64_t j = a.inj.row_ptr[r] + lane; j < a.inj.row_ptr[r + 1]; j += 32)
                s += a.inj.w[j] * a.res[a.inj.col[j] * (int64_t)a.nt + (a.m - 1)];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                int64_t loc = q - origin;
                int64_t dz = loc / L.px;
                acc[dz * TX + (loc - dz * L.px)] += s;
            }
        }
    }
    __syncthreads();
    const T wv = a.src.n ? a.wavelet[a.m - 1] : (T)0;
    const bool damped = damp_box(L, a.dw, x0, x0 + TX - 1, 0, 0, z0 + TZ - 1);
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j, lz = i / TX, lx = i - lz * TX;
        if (x0 + lx >= L.nx || z0 + lz >= L.nz) continue;
        const int64_t q = origin + lz * L.px + lx;
        // With an absorbing layer the buffers hold nu = mu / (1 + a): the transpose of
        // p^{n+1} = ((2 + K L) p^n - (1 - a) p^{n-1} + s) / (1 + a) is
        // mu^m = 2 nu^{m+1} - (1 - a) nu^{m+2} + L^T (K nu^{m+1}) + R^T res^{m-1}.
        const T av = damped ? damp_a<T>(L, a.dw, a.da, x0 + lx, 0, z0 + lz) : (T)0;
        T mu_new = (T)2 * mu_v[j] - ((T)1 - av) * mum_v[j] + acc[i];
        if (damped) mu_new = mu_new / ((T)1 + av);
        a.out[q] = mu_new;
        const T Kq = kh_v[j];
        if (Kq > (T)0) {
            // dt^2 c^2 (L p^{m-1}) = (1 + a) p^m - 2 p^{m-1} + (1 - a) p^{m-2} - s^{m-1}
            T d2 = (p0_v[j] - p1_v[j]) - (p1_v[j] - p2_v[j]);
            if (damped) d2 += av * (p0_v[j] - p2_v[j]);
            const T srcw = sw[i];
            d2 -= srcw * wv;
            a.grad[q] = g_v[j] + mu_new * (a.two_dt_over_h / sqrt(Kq)) * d2;
            if (a.gw && srcw != (T)0) atomicAdd(&a.gw[a.m - 1], srcw * mu_new);
        }
    }
}

template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256) k_adj2d(AdjArgs<T> a) {
    __shared__ __align__(16) T tile[TZ + 2 * H][TX + 8];     // K mu on the halo tile
    __shared__ __align__(16) T tmu[(TZ + 2 * H) * (TX + 8)];
    __shared__ T acc[TZ * TX];
    __shared__ T sw[TZ * TX];                      // source weights landing in the tile
    adj2d_tile<T, H, TX, TZ>(a, blockIdx.x, blockIdx.y, tile, tmu, acc, sw);
}

// Batched adjoint step m of segment [c, e) over many shots: block -> (shot, tile)
// by table.  mu^{m+1} / mu^{m+2} alternate between the shot's two buffers with
// the number of steps taken (nt - m); the segment buffer holds p^{c-1+j} in slot j.
template <typename T>
struct AdjBatch {
    AdjArgs<T> a;
    T* mu1;
    T* mu2;
    T* seg;               // segment buffer: (seg_len + 2) padded fields
};

template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256, 3) k_adj2d_batch(const AdjBatch<T>* __restrict__ shots,
                                                     const int64_t* __restrict__ tile0,
                                                     const int32_t* __restrict__ shot_of, int m, int j, int nt) {
    __shared__ __align__(16) T tile[TZ + 2 * H][TX + 8];
    __shared__ __align__(16) T tmu[(TZ + 2 * H) * (TX + 8)];
    __shared__ T acc[TZ * TX];
    __shared__ T sw[TZ * TX];
    const int64_t b = blockIdx.x;
    const int sh = shot_of[b];
    const AdjBatch<T>& B = shots[sh];
    AdjArgs<T> a = B.a;
    const bool even = ((nt - m) & 1) == 0;
    a.mu = even ? B.mu1 : B.mu2;
    a.mum = even ? B.mu2 : B.mu1;
    a.out = const_cast<T*>(a.mum);
    a.m = m;
    const int64_t tot = a.L.total;
    a.pm0 = B.seg + (int64_t)(j + 1) * tot;
    a.pm1 = B.seg + (int64_t)j * tot;
    a.pm2 = B.seg + (int64_t)(j - 1) * tot;
    const int64_t local = b - tile0[sh];
    const int64_t ntiles = a.opT.ntx * ((a.L.nz + TZ - 1) / TZ);
    if (local >= ntiles) return;   // uniform per block
    adj2d_tile<T, H, TX, TZ>(a, local % a.opT.ntx, local / a.opT.ntx, tile, tmu, acc, sw);
}

// ---------------------------------------------------------------------------
// setup kernels (coefficients formed in FP64, rounded once)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_leap_coef(Layout L, const T* vel, const uint8_t* mask, double dt_over_h, T* Kh) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % L.nx, r = i / L.nx, y = r % L.ny, z = r / L.ny;
        int64_t q = L.idx(x, y, z);
        double c = (double)vel[i] * dt_over_h;
        Kh[q] = mask[q] ? (T)(c * c) : (T)0;
    }
}

template <typename T>
__global__ void k_stag_coef(Layout L, const T* vel, const T* rho, const uint8_t* mp, const uint8_t* mvx,
                            const uint8_t* mvz, double dt, double inv_h, T* kp, T* bx, T* bz) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % L.nx, z = i / L.nx;
        int64_t q = L.idx(x, 0, z);
        double r0 = rho ? (double)rho[i] : 1.0;
        double c = (double)vel[i];
        kp[q] = mp[q] ? (T)(dt * r0 * c * c * inv_h) : (T)0;
        double rx = (rho && x + 1 < L.nx) ? (double)rho[i + 1] : r0;
        double rz = (rho && z + 1 < L.nz) ? (double)rho[i + L.nx] : r0;
        bx[q] = mvx[q] ? (T)(dt * 0.5 * (1.0 / r0 + 1.0 / rx) * inv_h) : (T)0;
        bz[q] = mvz[q] ? (T)(dt * 0.5 * (1.0 / r0 + 1.0 / rz) * inv_h) : (T)0;
    }
}

template <typename T>
__global__ void k_interp_setup(int n, const double* xyz, int ndim, double inv_h, Layout L, const uint8_t* mask,
                               double scale, int64_t* idx, T* w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t b[3] = {0, 0, 0};
        double fr[3] = {0, 0, 0};
        int64_t nn[3] = {L.nx, ndim == 3 ? L.ny : L.nz, L.nz};
        for (int a = 0; a < ndim; ++a) {
            double xi = xyz[(int64_t)i * ndim + a] * inv_h;
            b[a] = (int64_t)floor(xi);
            fr[a] = xi - (double)b[a];
        }
        for (int c = 0; c < 8; ++c) {
            double wt = 0.0;
            int64_t q = L.base;
            if (c < (1 << ndim)) {
                wt = 1.0;
                int64_t node[3] = {0, 0, 0};
                bool in = true;
                for (int a = 0; a < ndim; ++a) {
                    int bit = (c >> a) & 1;
                    node[a] = b[a] + bit;
                    wt *= bit ? fr[a] : 1.0 - fr[a];
                    if (node[a] < 0 || node[a] >= nn[a]) in = false;
                }
                if (in) {
                    q = ndim == 3 ? L.idx(node[0], node[1], node[2]) : L.idx(node[0], 0, node[1]);
                    if (mask && !mask[q]) wt = 0.0;
                } else {
                    wt = 0.0;
                }
                if (wt == 0.0) q = L.base;
            }
            idx[8 * (int64_t)i + c] = q;
            w[8 * (int64_t)i + c] = (T)(wt * scale);
        }
    }
}

template <typename T>
__global__ void k_unpad(Layout L, const T* pad, T* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % L.nx, r = i / L.nx, y = r % L.ny, z = r / L.ny;
        out[i] = pad[L.idx(x, y, z)];
    }
}

// ---------------------------------------------------------------------------
// stability checks
//   - every forward / adjoint run ends with a pass over its final fields; a
//     NaN or Inf sets bit 0 of a per-device status word that ib_sync_status
//     reports as IB_ERR_UNSTABLE (a non-finite value never leaves the leapfrog
//     or staggered recursion once it appears, so the final fields suffice);
//   - ib_stability runs the step kernels source-free from a random state and
//     renormalises every STAB_BLOCK steps: a power iteration on the one-step
//     map whose per-step growth estimates its spectral radius.
// ---------------------------------------------------------------------------
static __device__ int g_dev_status;

template <typename T>
__global__ void k_check_finite(int64_t n, const T* __restrict__ a, const T* __restrict__ b,
                               const T* __restrict__ c) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        bad |= !isfinite(a[i]);
        if (b) bad |= !isfinite(b[i]);
        if (c) bad |= !isfinite(c[i]);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&g_dev_status, 1);
}

// SplitMix64 output function (Steele, Lea & Flood, "Fast splittable
// pseudorandom number generators", 2014) as a counter-based generator
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// f[i] = f2[i] = uniform(-1, 1) where coef[i] != 0 (interior nodes), else 0
template <typename T>
__global__ void k_rand_fill(int64_t n, const T* __restrict__ coef, uint64_t seed, T* f, T* f2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = (T)0;
        if (coef[i] != (T)0) v = (T)((double)(splitmix64(seed * 0x632be59bd9b4e019ull + (uint64_t)i) >> 11) *
                                         (2.0 / 9007199254740992.0) - 1.0);
        f[i] = v;
        if (f2) f2[i] = v;
    }
}

// *out += sum of squares of a, b, c (nullable)
template <typename T>
__global__ void k_sumsq(int64_t n, const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ c,
                        double* out) {
    __shared__ double part[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = (double)a[i];
        s += x * x;
        if (b) {
            x = (double)b[i];
            s += x * x;
        }
        if (c) {
            x = (double)c[i];
            s += x * x;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(out, t);
    }
}

// divide a, b, c by sqrt(*sumsq); *logn = log sqrt(*sumsq)
template <typename T>
__global__ void k_rescale(int64_t n, T* a, T* b, T* c, const double* sumsq, double* logn) {
    const double nrm = sqrt(*sumsq);
    const T inv = (T)(nrm > 0.0 ? 1.0 / nrm : 0.0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a[i] *= inv;
        if (b) b[i] *= inv;
        if (c) c[i] *= inv;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *logn = log(nrm);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int grid1(int64_t n, int bs) {
    int64_t g = (n + bs - 1) / bs;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <class T>
    ib_status alloc(T** p, int64_t n, bool zero = false) {
        *p = nullptr;
        if (n <= 0) n = 1;
        IB_CUDA(cudaMallocAsync((void**)p, sizeof(T) * (size_t)n, s));
        ptrs.push_back(*p);
        if (zero) IB_CUDA(cudaMemsetAsync(*p, 0, sizeof(T) * (size_t)n, s));
        return IB_OK;
    }
};

// power-iteration probe of ib_stability: random start, renormalisation every
// STAB_BLOCK steps into slot k of the device arrays sums / logs
static const int STAB_BLOCK = 50;
struct Probe {
    uint64_t seed;
    int nslot;          // nt / STAB_BLOCK + 1 (slot 0: the initial norm)
    double* sums;       // [nslot], zeroed
    double* logs;       // [nslot]
};

// Renormalise the state (a, b, c) by its norm; `extra` (n_extra values, not part
// of the norm) holds quantities linear in the state that the next step reads --
// the staggered form's producer-side partial sums -- and is scaled alike.
template <typename T>
static ib_status probe_rescale(const Probe* pr, int slot, int64_t n, T* a, T* b, T* c, cudaStream_t s,
                               T* extra = nullptr, int64_t n_extra = 0) {
    k_sumsq<T><<<grid1(n, 256), 256, 0, s>>>(n, a, b, c, pr->sums + slot);
    k_rescale<T><<<grid1(n, 256), 256, 0, s>>>(n, a, b, c, pr->sums + slot, pr->logs + slot);
    ib_count_launch("setup");
    ib_count_launch("setup");
    if (extra && n_extra > 0) {
        k_rescale<T><<<grid1(n_extra, 256), 256, 0, s>>>(n_extra, extra, (T*)nullptr, (T*)nullptr,
                                                          pr->sums + slot, pr->logs + slot);
        ib_count_launch("setup");
    }
    IB_CHECK_LAUNCH("stability probe");
    return IB_OK;
}

template <typename T>
static ib_status check_finite(int64_t n, const T* a, const T* b, const T* c, cudaStream_t s) {
    k_check_finite<T><<<grid1(n, 256), 256, 0, s>>>(n, a, b, c);
    IB_CHECK_LAUNCH("k_check_finite");
    ib_count_launch("setup");
    return IB_OK;
}

template <typename T>
static void stencil_weights(int M, T w2o[5], T c1o[4]) {
    std::vector<double> w2 = ib_central_second(M);
    std::vector<double> c1 = ib_staggered_first(M);
    int H = M / 2;
    for (int k = 0; k < 5; ++k) w2o[k] = k <= H ? (T)w2[H + k] : (T)0;
    for (int k = 0; k < 4; ++k) c1o[k] = k < H ? (T)c1[H + k] : (T)0;   // offset +(k + 1/2)
}

template <typename T>
static TileView<T> tview(const TileBins* b) {
    TileView<T> v;
    memset(&v, 0, sizeof v);
    if (!b || b->nent == 0) return v;
    v.ptr = b->ent_ptr;
    v.loc = b->ent_loc;
    v.src = b->ent_src;
    v.w = (const T*)(sizeof(T) == 8 ? (const void*)b->ent_w64 : (const void*)b->ent_w32);
    v.ntx = b->ntx;
    return v;
}

static const int TX2 = 64, TZ2 = 8;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
static PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

static bool tma_enabled() {
    const char* e = getenv("IB_NO_TMA");
    return tma_encode_fn() != nullptr && !(e && e[0] == '1');
}

// 2D view of a padded FP32 3D field: rows of px elements; box (tw + 8) x (8 + 2H)
// (a plane of a tile tw wide with its halo) or, with tile_only, tw x 8 (a tile
// without halo)
static ib_status make_plane_map(CUtensorMap& tm, void* base, const Layout& L, bool tile_only = false,
                                uint32_t tw = 32) {
    cuuint64_t dims[2] = {(cuuint64_t)L.px, (cuuint64_t)(L.total / L.px)};
    cuuint64_t strides[1] = {(cuuint64_t)L.px * 4};
    cuuint32_t box[2] = {tile_only ? tw : tw + 8u, tile_only ? 8u : (cuuint32_t)(8 + 2 * L.H)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = tma_encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        ib_set_error("cuTensorMapEncodeTiled failed");
        return IB_ERR_CUDA;
    }
    return IB_OK;
}

static bool shot_damped(const ib_shot* sh) { return sh->damp_width > 0 && sh->damp_eta > 0.0; }

static ib_status check_shot(const ib_table* t, const ib_shot* sh, int precision, double dt, int nt,
                            bool need_traces = true) {
    if (!t || !sh) {
        ib_set_error("null table or shot");
        return IB_ERR_ARG;
    }
    if (precision != 32 && precision != 64) {
        ib_set_error("precision must be 32 or 64");
        return IB_ERR_ARG;
    }
    if (!(dt > 0.0) || nt < 1) {
        ib_set_error("dt must be positive and nt >= 1");
        return IB_ERR_ARG;
    }
    if (!sh->vel_dev || sh->nsrc < 0 || sh->nrec < 0 || (sh->nsrc && (!sh->src_dev || !sh->wavelet_dev)) ||
        (sh->nrec && (!sh->rec_dev || (need_traces && !sh->traces_dev)))) {
        ib_set_error("missing shot arrays");
        return IB_ERR_ARG;
    }
    if (!(sh->damp_eta >= 0.0) || sh->damp_width < 0 ||
        (shot_damped(sh) && 2 * (int64_t)sh->damp_width >= t->grid.n[0])) {
        ib_set_error("absorbing layer: damp_eta >= 0 and 0 <= damp_width < nx / 2 required");
        return IB_ERR_ARG;
    }
    if (sh->nsrc > 32) {
        // the step kernels spread each source over its 8 interpolation corners with
        // one thread per corner of a 256-thread block
        ib_set_error("at most 32 sources per shot");
        return IB_ERR_ARG;
    }
    return IB_OK;
}

template <typename T>
struct Geom {
    PointSet<T> src, rec;
};

// absorbing layer of a shot: width and a_max = eta_max dt / 2 (formed in FP64)
template <typename T>
static void set_damping(const ib_shot* sh, double dt, int& dw, T& da) {
    dw = shot_damped(sh) ? sh->damp_width : 0;
    da = dw ? (T)(0.5 * sh->damp_eta * dt) : (T)0;
}

template <typename T>
static ib_status setup_points(const ib_table* t, const ib_shot* sh, double scale, Scratch& S, Geom<T>& g) {
    const Layout& L = t->L;
    int d = t->grid.ndim;
    int64_t* si;
    T* sw;
    int64_t* ri;
    T* rw;
    TRY(S.alloc(&si, 8 * std::max(sh->nsrc, 1)));
    TRY(S.alloc(&sw, 8 * std::max(sh->nsrc, 1)));
    TRY(S.alloc(&ri, 8 * std::max(sh->nrec, 1)));
    TRY(S.alloc(&rw, 8 * std::max(sh->nrec, 1)));
    if (sh->nsrc) {
        k_interp_setup<T><<<grid1(sh->nsrc, 64), 64, 0, S.s>>>(sh->nsrc, sh->src_dev, d, 1.0 / t->grid.h, L,
                                                                t->mask_pad[0], scale, si, sw);
        ib_count_launch("setup");
    }
    if (sh->nrec) {
        k_interp_setup<T><<<grid1(sh->nrec, 64), 64, 0, S.s>>>(sh->nrec, sh->rec_dev, d, 1.0 / t->grid.h, L,
                                                                t->mask_pad[0], 1.0, ri, rw);
        ib_count_launch("setup");
    }
    IB_CHECK_LAUNCH("k_interp_setup");
    g.src = {sh->nsrc, si, sw};
    g.rec = {sh->nrec, ri, rw};
    return IB_OK;
}

// checkpoint slot k holds (p^{c_k}, p^{c_k - 1}), c_k = k * seg
static int64_t ckpt_seg(int nt, int n_ckpt) { return (nt + n_ckpt - 1) / n_ckpt; }

extern "C" int64_t ib_checkpoint_bytes(const ib_table* t, int32_t precision, int32_t nt, int32_t n_ckpt) {
    if (!t || n_ckpt < 1 || nt < 1) return 0;
    int64_t es = precision == 64 ? 8 : 4;
    return (int64_t)n_ckpt * 2 * t->L.total * es;
}

static const int STRIP_NSUB = 8, STRIP_D = 3;   // z-marched strips: 8 tiles of 64 x 8, 3 in flight

// One FP32 shot runs on strips when there are enough of them to fill the GPU
// (a strip is 8 tiles of work: on small grids the tile kernel keeps more blocks
// in flight).  IB_STRIP=0 / IB_STRIP=1 turn strips off / on whatever the size.
static bool use_strips(const Layout& L) {
    const int64_t nblk = ((L.nx + TX2 - 1) / TX2) * (((L.nz + TZ2 - 1) / TZ2 + STRIP_NSUB - 1) / STRIP_NSUB);
    const char* e = getenv("IB_STRIP");
    if (e && *e) return e[0] != '0';
    return nblk >= 1024;
}

template <typename T>
static void launch_leap2d(const StepArgs<T>& a, int H, dim3 grid, cudaStream_t s) {
    PROF_LAUNCH(kname<T>("leap2d_f32", "leap2d_f64"), s, {
        if (H == 1) k_leap2d<T, 1, TX2, TZ2><<<grid, 256, 0, s>>>(a);
        else if (H == 2) k_leap2d<T, 2, TX2, TZ2><<<grid, 256, 0, s>>>(a);
        else if (H == 3) k_leap2d<T, 3, TX2, TZ2><<<grid, 256, 0, s>>>(a);
        else k_leap2d<T, 4, TX2, TZ2><<<grid, 256, 0, s>>>(a);
    });
}

static void launch_leap2d_strip(const StepArgs<float>& a, int H, dim3 grid, cudaStream_t s) {
    PROF_LAUNCH("leap2d_strip_f32", s, {
        if (H == 1) k_leap2d_m<1, STRIP_NSUB, STRIP_D><<<grid, 256, 0, s>>>(a);
        else if (H == 2) k_leap2d_m<2, STRIP_NSUB, STRIP_D><<<grid, 256, 0, s>>>(a);
        else if (H == 3) k_leap2d_m<3, STRIP_NSUB, STRIP_D><<<grid, 256, 0, s>>>(a);
        else k_leap2d_m<4, STRIP_NSUB, STRIP_D><<<grid, 256, 0, s>>>(a);
    });
}

// ---------------------------------------------------------------------------
// Temporal blocking: two leapfrog steps per launch (2D, second order, FP32).
//
// A block owns a TX x TZ output tile.  It stages p^n on the tile grown by 2R
// ("region 2"), computes p^{n+1} on the tile grown by R ("region 1": standard
// stencil, the immersed-boundary rows that lie there, source, absorbing
// layer) and keeps it in shared memory, then computes p^{n+2} on the tile from
// it.  R >= M/2 and R >= the reach of every correction row, so both steps read
// shared memory only.  The ring of region 1 outside the tile is computed by the
// neighbouring blocks as well: 2 x (1 + 2R/TX)(1 + 2R/TZ)/2 stencils per point
// and step instead of 1, for DRAM traffic of p^n, p^{n-1}, K read and p^{n+1},
// p^{n+2} written per two steps (20 bytes per point, 10 per point and step,
// against 16 for one step per launch).  Outputs go to two further buffers:
// the neighbours still read p^n and p^{n-1} in their halos.
//
// Correction entries of a tile: every row in region 1, those inside the tile
// first (used by both steps), one int32 code per entry -- the row's position
// in region 1 (x, z: 8 bits each) and the column offset (dx, dz: int8 each) --
// and the FP32 weight.
// ---------------------------------------------------------------------------
struct TbArgs {
    Layout L;
    float w2[5];
    const float* pn;         // p^n
    const float* pm;         // p^{n-1}
    const float* Kh;
    float* out1;             // p^{n+1}
    float* out2;             // p^{n+2}
    const int32_t* ent_ptr;  // [2 ntiles + 1]: tile t has rows [2t, 2t+1) in the tile, [2t+1, 2t+2) in its ring
    const int32_t* ent_code;
    const float* ent_w;
    PointSet<float> src;
    const float* wavelet;
    int step;                // n (the launch advances n -> n + 2)
    PointSet<float> rec;
    float* traces;
    int nt;
    int dw;
    float da;
};

__device__ __forceinline__ void tb_decode(int32_t c, int& lx, int& lz, int& dx, int& dz) {
    lx = c & 0xff;
    lz = (c >> 8) & 0xff;
    dx = (int)(int8_t)((c >> 16) & 0xff);
    dz = (int)(int8_t)((c >> 24) & 0xff);
}

// dst[loc(e)] += w[e] * f[col(e)] for the entries [e0, e1): four chunks of 32
// entries in flight per warp, segmented warp sums (entries of a row are
// contiguous), one shared-memory atomic per row segment
template <class LocCol>
__device__ __forceinline__ void tb_entries(const TbArgs& a, int32_t e0, int32_t e1, LocCol lc, const float* f,
                                           float* dst, int tid) {
    constexpr int U = 4;
    const int lane = tid & 31;
    for (int32_t base = e0 + (tid & ~31) * U; base < e1; base += 256 * U) {
        int32_t loc[U];
        float val[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t e = base + u * 32 + lane;
            ok[u] = e < e1;
            int l = -1 - lane, col = 0;
            if (ok[u]) lc(a.ent_code[e], l, col);
            loc[u] = l;
            val[u] = ok[u] ? a.ent_w[e] * f[col] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) seg_add(dst, loc[u], val[u], ok[u], lane);
    }
}

// dst[(z - zr) W + (x - xr)] += w wv for the source corners in the W x Z box at
// (xr, zr) that are nodes of the model (corners in the zero padding are dropped,
// as the one-step kernels drop them)
__device__ __forceinline__ void tb_sources(const PointSet<float>& src, float wv, const Layout& L, int64_t xr,
                                           int64_t zr, int W, int Z, float* dst, int tid) {
    if (tid >= 8 * src.n) return;
    const float w = src.w[tid];
    if (w == 0.f) return;
    const int64_t rel = src.idx[tid] - L.base;
    const int64_t z = rel >= 0 ? rel / L.px : -((-rel + L.px - 1) / L.px);
    const int64_t x = rel - z * L.px;
    if (x >= L.nx || z < 0 || z >= L.nz) return;
    const int64_t lx = x - xr, lz = z - zr;
    if (lx >= 0 && lx < W && lz >= 0 && lz < Z) atomicAdd(&dst[lz * W + lx], w * wv);
}

template <int R, int TX, int TZ>
struct TbShape {
    static constexpr int W1 = TX + 2 * R, Z1 = TZ + 2 * R, W2 = TX + 4 * R, Z2 = TZ + 4 * R;
    static constexpr size_t smem = sizeof(float) * ((size_t)W2 * Z2 + 2 * (size_t)W1 * Z1);
    static_assert(W1 <= 256 && Z1 <= 256, "region-1 positions take 8 bits per axis");
    static_assert((TX * TZ) % 256 == 0, "whole tile points per thread");
};

template <int H, int R, int TX, int TZ>
__global__ void __launch_bounds__(256) k_leap2d_tb2(TbArgs a) {
    using S = TbShape<R, TX, TZ>;
    constexpr int W1 = S::W1, Z1 = S::Z1, W2 = S::W2, Z2 = S::Z2;
    extern __shared__ float tb_sm[];
    float* P0 = tb_sm;             // p^n on region 2
    float* P1 = P0 + W2 * Z2;      // p^{n+1} on region 1
    float* A = P1 + W1 * Z1;       // accumulator (region 1, then the tile)
    const int tid = threadIdx.x;
    const Layout& L = a.L;
    const int64_t x0 = (int64_t)blockIdx.x * TX, z0 = (int64_t)blockIdx.y * TZ;
    const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    // trace columns n - 1 (p^n) and n - 2 (p^{n-1}): both inputs of this launch
    {
        const int64_t gid = tile * 256 + tid, stride = launch_threads();
        record_receivers(a.rec, a.pn, a.traces, a.nt, a.step - 1, gid, stride);
        record_receivers(a.rec, a.pm, a.traces, a.nt, a.step - 2, gid, stride);
    }
    for (int i = tid; i < W2 * Z2; i += 256) {
        const int lz = i / W2, lx = i - lz * W2;
        const int64_t x = x0 + lx - 2 * R, z = z0 + lz - 2 * R;
        const bool ok = x >= 0 && x < L.nx && z >= 0 && z < L.nz;
        cp_async<4>(&P0[i], ok ? a.pn + L.base + z * L.px + x : a.pn, ok);
    }
    cp_async_commit();
    const int32_t e0 = a.ent_ptr[2 * tile], em = a.ent_ptr[2 * tile + 1], e1 = a.ent_ptr[2 * tile + 2];
    cp_async_wait_all();
    __syncthreads();
    // ---- step n -> n + 1 on region 1
    for (int i = tid; i < W1 * Z1; i += 256) {
        const int lz = i / W1, lx = i - lz * W1;
        const float* q = P0 + (lz + R) * W2 + lx + R;
        const float c = q[0];
        float s = 0.f;
#pragma unroll
        for (int k = 1; k <= H; ++k)
            s += a.w2[k] * (((q[k] - c) + (q[-k] - c)) + ((q[k * W2] - c) + (q[-k * W2] - c)));
        A[i] = s;
    }
    __syncthreads();
    if (e1 > e0)
        tb_entries(
            a, e0, e1,
            [](int32_t code, int& loc, int& col) {
                int lx, lz, dx, dz;
                tb_decode(code, lx, lz, dx, dz);
                loc = lz * W1 + lx;
                col = (lz + R + dz) * W2 + lx + R + dx;
            },
            P0, A, tid);
    __syncthreads();
    // update (A keeps p^{n-1} for the absorbing layer), then the source
    for (int i = tid; i < W1 * Z1; i += 256) {
        const int lz = i / W1, lx = i - lz * W1;
        const int64_t x = x0 + lx - R, z = z0 + lz - R;
        float u = 0.f, pmv = 0.f;
        if (x >= 0 && x < L.nx && z >= 0 && z < L.nz) {
            const int64_t q = L.base + z * L.px + x;
            const float c = P0[(lz + R) * W2 + lx + R];
            pmv = a.pm[q];
            u = c + ((c - pmv) + a.Kh[q] * A[i]);
        }
        P1[i] = u;
        A[i] = pmv;
    }
    __syncthreads();
    if (a.src.n) {
        tb_sources(a.src, a.wavelet[a.step], L, x0 - R, z0 - R, W1, Z1, P1, tid);
        __syncthreads();
    }
    if (damp_box(L, a.dw, x0 - R, x0 + TX - 1 + R, 0, 0, z0 + TZ - 1 + R)) {
        for (int i = tid; i < W1 * Z1; i += 256) {
            const int lz = i / W1, lx = i - lz * W1;
            const int64_t x = x0 + lx - R, z = z0 + lz - R;
            if (x >= 0 && x < L.nx && z >= 0 && z < L.nz)
                P1[i] -= damp_g<float>(L, a.dw, a.da, x, 0, z) * (P1[i] - A[i]);
        }
    }
    __syncthreads();
    // ---- step n + 1 -> n + 2 on the tile
    constexpr int PT = TX * TZ / 256;
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j, lz = i / TX, lx = i - lz * TX;
        const float* q = P1 + (lz + R) * W1 + lx + R;
        const float c = q[0];
        float s = 0.f;
#pragma unroll
        for (int k = 1; k <= H; ++k)
            s += a.w2[k] * (((q[k] - c) + (q[-k] - c)) + ((q[k * W1] - c) + (q[-k * W1] - c)));
        A[i] = s;
    }
    __syncthreads();
    if (em > e0)
        tb_entries(
            a, e0, em,
            [](int32_t code, int& loc, int& col) {
                int lx, lz, dx, dz;
                tb_decode(code, lx, lz, dx, dz);
                loc = (lz - R) * TX + lx - R;
                col = (lz + dz) * W1 + lx + dx;
            },
            P1, A, tid);
    __syncthreads();
    float uv[PT];
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j, lz = i / TX, lx = i - lz * TX;
        const int64_t x = x0 + lx, z = z0 + lz;
        uv[j] = 0.f;
        if (x < L.nx && z < L.nz) {
            const int64_t q = L.base + z * L.px + x;
            const float c = P1[(lz + R) * W1 + lx + R];
            const float pmv = P0[(lz + 2 * R) * W2 + lx + 2 * R];
            uv[j] = c + ((c - pmv) + a.Kh[q] * A[i]);
            a.out1[q] = c;
        }
    }
    if (a.src.n) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PT; ++j) A[tid + 256 * j] = uv[j];
        __syncthreads();
        tb_sources(a.src, a.wavelet[a.step + 1], L, x0, z0, TX, TZ, A, tid);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PT; ++j) uv[j] = A[tid + 256 * j];
    }
    const bool damped = damp_box(L, a.dw, x0, x0 + TX - 1, 0, 0, z0 + TZ - 1);
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int i = tid + 256 * j, lz = i / TX, lx = i - lz * TX;
        const int64_t x = x0 + lx, z = z0 + lz;
        if (x >= L.nx || z >= L.nz) continue;
        float u = uv[j];
        if (damped) {
            const float pmv = P0[(lz + 2 * R) * W2 + lx + 2 * R];
            u -= damp_g<float>(L, a.dw, a.da, x, 0, z) * (u - pmv);
        }
        a.out2[L.base + z * L.px + x] = u;
    }
}

static const int TBX = 64, TBZ = 32;

// Correction entries of the two-step kernel for region margin R, cached in the
// table's bins of operator 0 (key tx = TBX, ty = -R, tz = TBZ).  *ok = false
// when a correction reaches further than R (the one-step kernels run then).
static ib_status tb_bins(ib_table* t, int R, TileBins* out, bool* ok) {
    IbOp& op = t->ops[0];
    for (const TileBins& b : op.bins)
        if (b.tx == TBX && b.ty == -R && b.tz == TBZ) {
            *out = b;
            *ok = b.nent >= 0;
            return IB_OK;
        }
    const Layout& L = t->L;
    const int64_t nr = op.nrows, nnz = op.nnz;
    std::vector<int64_t> lin(nr), rp(nr + 1, 0);
    std::vector<int32_t> code(nnz);
    std::vector<float> w(nnz);
    if (nr) {
        IB_CUDA(cudaMemcpy(lin.data(), op.row_lin, 8 * nr, cudaMemcpyDeviceToHost));
        IB_CUDA(cudaMemcpy(rp.data(), op.row_ptr, 8 * (nr + 1), cudaMemcpyDeviceToHost));
    }
    if (nnz) {
        IB_CUDA(cudaMemcpy(code.data(), op.col_code, 4 * nnz, cudaMemcpyDeviceToHost));
        IB_CUDA(cudaMemcpy(w.data(), op.w32, 4 * nnz, cudaMemcpyDeviceToHost));
    }
    TileBins b;
    b.tx = TBX;
    b.ty = -R;
    b.tz = TBZ;
    b.ntx = (L.nx + TBX - 1) / TBX;
    b.nty = 1;
    const int64_t ntz = (L.nz + TBZ - 1) / TBZ;
    b.ntiles = b.ntx * ntz;
    bool fits = true;
    for (int64_t e = 0; e < nnz && fits; ++e) {
        int dx, dy, dz;
        unpack_off(code[e], dx, dy, dz);
        fits = std::abs(dx) <= R && std::abs(dy) <= R;
    }
    if (!fits) {   // remembered, so that the check runs once per table
        b.nent = -1;
        op.bins.push_back(b);
        *out = b;
        *ok = false;
        return IB_OK;
    }
    // visit (row, tile, in-tile?) for every tile whose region 1 holds the row
    auto each = [&](auto&& f) {
        for (int64_t r = 0; r < nr; ++r) {
            const int64_t x = lin[r] % L.nx, z = lin[r] / L.nx;
            for (int64_t bz = std::max<int64_t>(0, (z - R) / TBZ - 1); bz <= std::min(ntz - 1, (z + R) / TBZ); ++bz) {
                if (z < bz * TBZ - R || z > bz * TBZ + TBZ - 1 + R) continue;
                for (int64_t bx = std::max<int64_t>(0, (x - R) / TBX - 1); bx <= std::min(b.ntx - 1, (x + R) / TBX);
                     ++bx) {
                    if (x < bx * TBX - R || x > bx * TBX + TBX - 1 + R) continue;
                    const bool in = x >= bx * TBX && x < bx * TBX + TBX && z >= bz * TBZ && z < bz * TBZ + TBZ;
                    f(r, x, z, bx, bz, in);
                }
            }
        }
    };
    std::vector<int64_t> cnt(2 * b.ntiles, 0);
    each([&](int64_t r, int64_t, int64_t, int64_t bx, int64_t bz, bool in) {
        cnt[2 * (bz * b.ntx + bx) + (in ? 0 : 1)] += rp[r + 1] - rp[r];
    });
    std::vector<int32_t> ptr(2 * b.ntiles + 1, 0);
    int64_t tot = 0;
    for (int64_t i = 0; i < 2 * b.ntiles; ++i) {
        ptr[i] = (int32_t)tot;
        tot += cnt[i];
    }
    if (tot >= INT32_MAX) {
        ib_set_error("two-step correction list exceeds 2^31 entries");
        return IB_ERR_ARG;
    }
    ptr[2 * b.ntiles] = (int32_t)tot;
    std::vector<int32_t> ecode(std::max<int64_t>(tot, 1));
    std::vector<float> ew(std::max<int64_t>(tot, 1));
    std::vector<int64_t> cur(ptr.begin(), ptr.end() - 1);
    each([&](int64_t r, int64_t x, int64_t z, int64_t bx, int64_t bz, bool in) {
        const uint32_t lx = (uint32_t)(x - (bx * TBX - R)), lz = (uint32_t)(z - (bz * TBZ - R));
        int64_t& c = cur[2 * (bz * b.ntx + bx) + (in ? 0 : 1)];
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e, ++c) {
            int dx, dy, dz;
            unpack_off(code[e], dx, dy, dz);
            ecode[c] = (int32_t)(lx | lz << 8 | (uint32_t)(dx & 0xff) << 16 | (uint32_t)(dy & 0xff) << 24);
            ew[c] = w[e];
        }
    });
    b.nent = tot;
    auto up = [](auto** d, const auto& v) -> ib_status {
        IB_CUDA(cudaMalloc((void**)d, sizeof(v[0]) * v.size()));
        IB_CUDA(cudaMemcpy(*d, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice));
        return IB_OK;
    };
    ib_status st = up(&b.ent_ptr, ptr);
    if (st == IB_OK) st = up(&b.ent_loc, ecode);
    if (st == IB_OK) st = up(&b.ent_w32, ew);
    if (st != IB_OK) {
        ib_free_bins(b);
        return st;
    }
    op.bins.push_back(b);
    *out = b;
    *ok = true;
    return IB_OK;
}

// IB_TEMPORAL_BLOCK=0 / 1 turns the two-step kernel off / on
static bool tb_enabled() {
    const char* e = getenv("IB_TEMPORAL_BLOCK");
    return e && e[0] == '1';
}

template <int H, int R>
static void launch_tb2_hr(const TbArgs& a, dim3 grid, cudaStream_t s) {
    using Sh = TbShape<R, TBX, TBZ>;
    static const bool attr = (cudaFuncSetAttribute(k_leap2d_tb2<H, R, TBX, TBZ>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem),
                              true);
    (void)attr;
    k_leap2d_tb2<H, R, TBX, TBZ><<<grid, 256, Sh::smem, s>>>(a);
}
template <int R>
static void launch_tb2_r(const TbArgs& a, int H, dim3 grid, cudaStream_t s) {
    if (H == 1) launch_tb2_hr<1, R>(a, grid, s);
    else if (H == 2) launch_tb2_hr<2, R>(a, grid, s);
    else if (H == 3) launch_tb2_hr<3, R>(a, grid, s);
    else launch_tb2_hr<4, R>(a, grid, s);
}
// region margins the two-step kernel is built for (R >= M/2 and >= the reach)
static const int TB_MARGINS[2] = {4, 6};
static void launch_tb2(const TbArgs& a, int H, int R, dim3 grid, cudaStream_t s) {
    PROF_LAUNCH("leap2d_tb2_f32", s, {
        if (R == 4) launch_tb2_r<4>(a, H, grid, s);
        else launch_tb2_r<6>(a, H, grid, s);
    });
}

// Single FP32 shots on strips use 64 x 16 tiles with two columns per thread
// (IB_STRIP4=0 selects the 64 x 8 strips): 134 against 176 us per step at
// 8192 x 4096, order 8.
static bool strip4_enabled() {
    const char* e = getenv("IB_STRIP4");
    return !(e && e[0] == '0');
}

template <int H>
static void launch_strip4_h(const StepArgs<float>& a, dim3 grid, cudaStream_t s) {
    constexpr size_t sm = Strip4<H, 4, 2>::FLOATS * sizeof(float);
    static const bool attr = (cudaFuncSetAttribute(k_leap2d_m4<H, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sm),
                              true);
    (void)attr;
    k_leap2d_m4<H, 4, 2><<<grid, 256, sm, s>>>(a);
}
static void launch_leap2d_strip4(const StepArgs<float>& a, int H, dim3 grid, cudaStream_t s) {
    PROF_LAUNCH("leap2d_strip_f32", s, {
        if (H == 1) launch_strip4_h<1>(a, grid, s);
        else if (H == 2) launch_strip4_h<2>(a, grid, s);
        else if (H == 3) launch_strip4_h<3>(a, grid, s);
        else launch_strip4_h<4>(a, grid, s);
    });
}

template <typename T>
static ib_status forward_2nd(ib_table* t, const ib_shot* sh, double dt, int nt, void* ckpt, int n_ckpt,
                             cudaStream_t s, const Probe* probe = nullptr) {
    const Layout& L = t->L;
    const int d = t->grid.ndim;
    const int M = t->opts.space_order;
    const int H = M / 2;
    Scratch S(s);
    T *p0, *p1, *Kh;
    TRY(S.alloc(&p0, L.total, true));
    TRY(S.alloc(&p1, L.total, true));
    TRY(S.alloc(&Kh, L.total, true));
    k_leap_coef<T><<<grid1(L.N, 256), 256, 0, s>>>(L, (const T*)sh->vel_dev, t->mask_pad[0], dt / t->grid.h, Kh);
    IB_CHECK_LAUNCH("k_leap_coef");
    ib_count_launch("setup");
    if (probe) {   // p^0 = p^{-1} = random on interior nodes, normalised
        k_rand_fill<T><<<grid1(L.total, 256), 256, 0, s>>>(L.total, Kh, probe->seed, p0, p1);
        IB_CHECK_LAUNCH("k_rand_fill");
        TRY(probe_rescale<T>(probe, 0, L.total, p0, p1, (T*)nullptr, s));
    }
    Geom<T> g;
    TRY(setup_points<T>(t, sh, dt * dt / pow(t->grid.h, d), S, g));
    const TileBins* bins = nullptr;
    if (d == 2) TRY(ib_table_bins(t, 0, false, TX2, 1, TZ2, &bins, s));
    else TRY(ib_table_bins(t, 0, false, 32, 8, 1, &bins, s));
    StepArgs<T> a;
    memset(&a, 0, sizeof a);
    a.L = L;
    {
        T c1u[4];
        stencil_weights<T>(M, a.w2, c1u);
    }
    a.Kh = Kh;
    a.op = tview<T>(bins);
    a.src = g.src;
    a.wavelet = (const T*)sh->wavelet_dev;
    a.rec = g.rec;
    a.traces = (T*)sh->traces_dev;
    a.nt = nt;
    set_damping<T>(sh, dt, a.dw, a.da);
    const int64_t seg = ckpt ? ckpt_seg(nt, n_ckpt) : 0;
    T* cur = p0;   // p^n
    T* prev = p1;  // p^{n-1}
    dim3 grid2((unsigned)((L.nx + TX2 - 1) / TX2), (unsigned)((L.nz + TZ2 - 1) / TZ2));
    const bool strips = d == 2 && sizeof(T) == 4 && use_strips(L);
    // strips of 64 x 16 tiles, two columns per thread (default; IB_STRIP4=0: 64 x 8)
    const bool strip4 = strips && strip4_enabled();
    StepArgs<T> a4 = a;
    dim3 grid4((unsigned)((L.nx + 63) / 64), (unsigned)(((L.nz + 15) / 16 + 3) / 4));
    if (strip4) {
        const TileBins* b4 = nullptr;
        TRY(ib_table_bins(t, 0, false, 64, 1, 16, &b4, s));
        a4.op = tview<T>(b4);
    }
    // two steps per launch (FP32 2D; not with checkpoints or the stability probe)
    int tbR = 0;
    TileBins tbb;
    float *tb_o1 = nullptr, *tb_o2 = nullptr;
    if (d == 2 && sizeof(T) == 4 && !ckpt && !probe && nt >= 2 && tb_enabled()) {
        for (int R : TB_MARGINS) {
            if (R < H) continue;
            bool ok = false;
            TRY(tb_bins(t, R, &tbb, &ok));
            if (ok) {
                tbR = R;
                break;
            }
        }
        if (tbR) {
            TRY(S.alloc(&tb_o1, L.total, true));
            TRY(S.alloc(&tb_o2, L.total, true));
        }
    }
    dim3 grids((unsigned)((L.nx + TX2 - 1) / TX2),
               (unsigned)(((L.nz + TZ2 - 1) / TZ2 + STRIP_NSUB - 1) / STRIP_NSUB));
    // planes per 3D block (IB_ZCHUNK overrides it for tuning)
    int zchunk = 32;
    if (const char* e = getenv("IB_ZCHUNK")) zchunk = std::max(1, atoi(e));
    dim3 grid3((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8), (unsigned)((L.nz + zchunk - 1) / zchunk));
    const int64_t nty3 = (L.ny + 7) / 8;
    // FP32 3D: TMA-staged planes of p (with halo) and tiles of p_prev and K (one
    // tensor map of each kind per buffer), compact correction rows
    CUtensorMap tmap[2], tmtile[2], tmK;
    Rows3 rows3;
    memset(&rows3, 0, sizeof rows3);
    const uint16_t* code16 = nullptr;
    int* err = nullptr;
    const bool use_tma = d == 3 && sizeof(T) == 4 && tma_enabled();
    // x-pair kernel (64 x 8 tiles; IB_TMA3_PAIRS=0 selects the 32 x 8 kernel)
    bool pairs = false;
    // correction pass: entries in flight per lane, 4 (IB_ADD3_U=8 selects 8: at
    // 512^2 x 384, order 8, 150 us per launch against 141 us with 4)
    int add3_u = 4;
    if (const char* e = getenv("IB_ADD3_U")) add3_u = atoi(e) == 8 ? 8 : 4;
    if (use_tma) {
        const char* fe = getenv("IB_FUSED3");
        const char* pe = getenv("IB_TMA3_PAIRS");
        pairs = !(fe && fe[0] == '1') && !(pe && pe[0] == '0');
        const uint32_t tw = pairs ? 64 : 32;
        TRY(make_plane_map(tmap[0], (void*)p0, L, false, tw));
        TRY(make_plane_map(tmap[1], (void*)p1, L, false, tw));
        TRY(make_plane_map(tmtile[0], (void*)p0, L, true, tw));
        TRY(make_plane_map(tmtile[1], (void*)p1, L, true, tw));
        TRY(make_plane_map(tmK, (void*)Kh, L, true, tw));
        TRY(S.alloc(&err, 1, true));
        // corrections: fused into the step kernel (IB_FUSED3=1) or added by k_ib_add3
        if (fe && fe[0] == '1') {
            if (bins && bins->nent > 0) {
                rows3.ptr = bins->ent_ptr;
                rows3.slot = bins->ent_slot;
                rows3.code = bins->ent_code;
                rows3.w = bins->ent_w32;
            }
        } else if (t->ops[0].nrows > 0) {
            TRY(ib_table_code16(t, 0, &code16, s));
        }
    }
    int n0 = 0;
    if (tbR) {
        TbArgs ta;
        memset(&ta, 0, sizeof ta);
        ta.L = L;
        for (int k = 0; k < 5; ++k) ta.w2[k] = (float)a.w2[k];
        ta.Kh = (const float*)Kh;
        ta.ent_ptr = tbb.ent_ptr;
        ta.ent_code = tbb.ent_loc;
        ta.ent_w = tbb.ent_w32;
        ta.src = *reinterpret_cast<const PointSet<float>*>(&g.src);
        ta.wavelet = (const float*)sh->wavelet_dev;
        ta.rec = *reinterpret_cast<const PointSet<float>*>(&g.rec);
        ta.traces = (float*)sh->traces_dev;
        ta.nt = nt;
        ta.dw = a.dw;
        ta.da = (float)a.da;
        dim3 gtb((unsigned)((L.nx + TBX - 1) / TBX), (unsigned)((L.nz + TBZ - 1) / TBZ));
        float *pc = (float*)cur, *pp = (float*)prev;
        for (; n0 + 2 <= nt; n0 += 2) {
            ta.pn = pc;
            ta.pm = pp;
            ta.out1 = tb_o1;
            ta.out2 = tb_o2;
            ta.step = n0;
            launch_tb2(ta, H, tbR, gtb, s);
            IB_CHECK_LAUNCH("two-step leapfrog");
            // p^{n+1}, p^{n+2} become (prev, cur); the old pair takes the next outputs
            tb_o1 = pp;
            tb_o2 = pc;
            pp = ta.out1;
            pc = ta.out2;
        }
        cur = (T*)pc;
        prev = (T*)pp;
        if (g.rec.n) {   // trace column n - 2 (p^{n-1}): the launches recorded columns up to n - 3
            k_receivers<T><<<grid1(g.rec.n, 256), 256, 0, s>>>(g.rec, prev, (T*)sh->traces_dev, nt, n0 - 2);
            IB_CHECK_LAUNCH("k_receivers");
            ib_count_launch("setup");
        }
    }
    for (int n = n0; n < nt; ++n) {
        if (ckpt && n % seg == 0) {
            T* slot = (T*)ckpt + (int64_t)(n / seg) * 2 * L.total;
            IB_CUDA(cudaMemcpyAsync(slot, cur, sizeof(T) * L.total, cudaMemcpyDeviceToDevice, s));
            IB_CUDA(cudaMemcpyAsync(slot + L.total, prev, sizeof(T) * L.total, cudaMemcpyDeviceToDevice, s));
        }
        a.p = cur;
        a.pm = prev;
        a.out = prev;
        a.step = n;
        a.rec_step = n - 1;
        if (strip4) {
            a4.p = a.p;
            a4.pm = a.pm;
            a4.out = a.out;
            a4.step = a.step;
            a4.rec_step = a.rec_step;
            launch_leap2d_strip4(*reinterpret_cast<const StepArgs<float>*>(&a4), H, grid4, s);
        } else if (strips) {
            launch_leap2d_strip(*reinterpret_cast<const StepArgs<float>*>(&a), H, grids, s);
        } else if (d == 2) {
            launch_leap2d<T>(a, H, grid2, s);
        } else if (use_tma) {
            dim3 blk(32, 8);
            const CUtensorMap& tmc = (cur == p0) ? tmap[0] : tmap[1];
            const CUtensorMap& tmm = (cur == p0) ? tmtile[1] : tmtile[0];   // p_prev: the other buffer
            PROF_LAUNCH("leap3d_tma_f32", s, {
                const StepArgs<float>& af = *reinterpret_cast<const StepArgs<float>*>(&a);
                if (pairs) {
                    dim3 gp((unsigned)((L.nx + 63) / 64), grid3.y, grid3.z);
                    if (H == 1) launch_leap3d_tma2<1>(af, tmc, tmm, tmK, zchunk, err, gp, s);
                    else if (H == 2) launch_leap3d_tma2<2>(af, tmc, tmm, tmK, zchunk, err, gp, s);
                    else if (H == 3) launch_leap3d_tma2<3>(af, tmc, tmm, tmK, zchunk, err, gp, s);
                    else launch_leap3d_tma2<4>(af, tmc, tmm, tmK, zchunk, err, gp, s);
                } else if (H == 1) launch_leap3d_tma<1>(af, tmc, tmm, tmK, rows3, zchunk, nty3, err, grid3, s);
                else if (H == 2) launch_leap3d_tma<2>(af, tmc, tmm, tmK, rows3, zchunk, nty3, err, grid3, s);
                else if (H == 3) launch_leap3d_tma<3>(af, tmc, tmm, tmK, rows3, zchunk, nty3, err, grid3, s);
                else launch_leap3d_tma<4>(af, tmc, tmm, tmK, rows3, zchunk, nty3, err, grid3, s);
            });
            if (code16) {
                const IbOp& op = t->ops[0];
                PROF_LAUNCH("ib_add3_f32", s, {
                    if (add3_u == 4)
                        k_ib_add3<4><<<grid1(op.nrows * 32, 256), 256, 0, s>>>(
                            op.nrows, op.row_pad, op.row_ptr, code16, op.w32, (const float*)a.p, (const float*)Kh,
                            (float*)a.out, L, a.dw, (float)a.da);
                    else
                        k_ib_add3<8><<<grid1(op.nrows * 32, 256), 256, 0, s>>>(
                            op.nrows, op.row_pad, op.row_ptr, code16, op.w32, (const float*)a.p, (const float*)Kh,
                            (float*)a.out, L, a.dw, (float)a.da);
                });
            }
        } else {
            dim3 blk(32, 8);
            PROF_LAUNCH(kname<T>("leap3d_f32", "leap3d_f64"), s, {
                if (H == 1) k_leap3d<T, 1><<<grid3, blk, 0, s>>>(a, zchunk, nty3);
                else if (H == 2) k_leap3d<T, 2><<<grid3, blk, 0, s>>>(a, zchunk, nty3);
                else if (H == 3) k_leap3d<T, 3><<<grid3, blk, 0, s>>>(a, zchunk, nty3);
                else k_leap3d<T, 4><<<grid3, blk, 0, s>>>(a, zchunk, nty3);
            });
        }
        IB_CHECK_LAUNCH("leapfrog step");
        std::swap(cur, prev);
        if (probe && (n + 1) % STAB_BLOCK == 0)
            TRY(probe_rescale<T>(probe, (n + 1) / STAB_BLOCK, L.total, cur, prev, (T*)nullptr, s));
    }
    if (g.rec.n) {
        k_receivers<T><<<grid1(g.rec.n, 256), 256, 0, s>>>(g.rec, cur, (T*)sh->traces_dev, nt, nt - 1);
        IB_CHECK_LAUNCH("k_receivers");
        ib_count_launch("setup");
    }
    if (!probe) TRY(check_finite<T>(L.total, cur, prev, (const T*)nullptr, s));
    if (use_tma) {
        int herr = 0;
        IB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        IB_CUDA(cudaStreamSynchronize(s));
        if (herr) {
            ib_set_error("a bounded TMA wait in the 3D step timed out");
            return IB_ERR_TIMEOUT;
        }
    }
    return IB_OK;
}

// Staggered step tiles: 64 x 32 (FP32) or 64 x 16 (FP64) nodes; at most
// STAG_MAXQ partial sums produced per tile.
static const int STAG_TX = 64, STAG_MAXQ = 1024;
static_assert(STAG_TX * 32 <= 2048 && STAG_MAXQ <= (1 << 20), "packed producer entries: 11-bit slot, 20-bit position");
template <typename T> struct StagTile { static const int TZ = 16, STG = 2048; };
template <> struct StagTile<double> { static const int TZ = 16, STG = 512; };

struct PlanOp {
    int op;       // consumer operator
    int target;   // accumulator of the consumer kernel (0: a_x / p, 1: a_z)
    int field;    // producer field of its columns (0: v_x / p, 1: v_z)
};

// Split the rows of the consumer operators by producer tile (see StagPlan):
// fills the consumer side of `cons` and the producer side of `prod`.
template <typename T>
static ib_status build_stag_plan(ib_table* t, const std::vector<PlanOp>& ops, int TZ, Scratch& S,
                                 StagPlan<T>& cons, StagPlan<T>& prod, cudaStream_t s) {
    const Layout& L = t->L;
    const int64_t ntx = (L.nx + STAG_TX - 1) / STAG_TX, ntz = (L.nz + TZ - 1) / TZ, ntiles = ntx * ntz;
    struct Ent {
        int32_t row, ptile, slot, field;
        double w;
    };
    struct Row {
        int32_t ctile, cslot;   // consumer tile and target << 24 | slot
    };
    std::vector<Ent> ent;
    std::vector<Row> rows;
    {
        int64_t nnz = 0, nr = 0;
        for (const PlanOp& po : ops) {
            nnz += t->ops[po.op].nnz;
            nr += t->ops[po.op].nrows;
        }
        ent.reserve(nnz);
        rows.reserve(nr);
    }
    for (const PlanOp& po : ops) {
        const IbOp& op = t->ops[po.op];
        const int64_t nr = op.nrows, nz = op.nnz;
        std::vector<int64_t> lin(nr), rp(nr + 1);
        std::vector<int32_t> code(nz);
        std::vector<double> w(nz);
        if (nr) {
            IB_CUDA(cudaMemcpy(lin.data(), op.row_lin, 8 * nr, cudaMemcpyDeviceToHost));
            IB_CUDA(cudaMemcpy(rp.data(), op.row_ptr, 8 * (nr + 1), cudaMemcpyDeviceToHost));
        }
        if (nz) {
            IB_CUDA(cudaMemcpy(code.data(), op.col_code, 4 * nz, cudaMemcpyDeviceToHost));
            IB_CUDA(cudaMemcpy(w.data(), op.w64, 8 * nz, cudaMemcpyDeviceToHost));
        }
        for (int64_t r = 0; r < nr; ++r) {
            const int64_t x = lin[r] % L.nx, z = lin[r] / L.nx;
            const int32_t key = (int32_t)rows.size();
            rows.push_back({(int32_t)((z / TZ) * ntx + x / STAG_TX),
                            (int32_t)(po.target << 24 | ((z % TZ) * STAG_TX + x % STAG_TX))});
            for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
                int dx, dy, dz;
                unpack_off(code[e], dx, dy, dz);
                const int64_t cx = x + dx, cz = z + dy;
                if (cx < 0 || cx >= L.nx || cz < 0 || cz >= L.nz) {
                    ib_set_error("correction column outside the grid");
                    return IB_ERR_STATE;
                }
                ent.push_back({key, (int32_t)((cz / TZ) * ntx + cx / STAG_TX),
                               (int32_t)((cz % TZ) * STAG_TX + cx % STAG_TX), po.field, w[e]});
            }
        }
    }
    // partial ids: one per (row, producer tile), numbered row by row.  Entries
    // arrive grouped by row; regroup each row's entries by producer tile (a row
    // spans a few tiles), keeping their order within a tile.
    const int64_t nrow = (int64_t)rows.size(), nent = (int64_t)ent.size();
    {
        std::vector<Ent> tmp;
        std::vector<int32_t> tiles;
        for (int64_t i = 0; i < nent;) {
            int64_t j = i;
            tiles.clear();
            for (; j < nent && ent[j].row == ent[i].row; ++j)
                if (std::find(tiles.begin(), tiles.end(), ent[j].ptile) == tiles.end()) tiles.push_back(ent[j].ptile);
            if (tiles.size() > 1) {
                std::sort(tiles.begin(), tiles.end());
                tmp.clear();
                for (int32_t tl : tiles)
                    for (int64_t k = i; k < j; ++k)
                        if (ent[k].ptile == tl) tmp.push_back(ent[k]);
                std::copy(tmp.begin(), tmp.end(), ent.begin() + i);
            }
            i = j;
        }
    }
    std::vector<int32_t> pid(nent), rank(nent), rpb(nrow, 0), rpe(nrow, 0);
    int32_t npid = 0;
    for (int64_t i = 0; i < nent; ++i) {
        const bool new_row = i == 0 || ent[i].row != ent[i - 1].row;
        if (new_row || ent[i].ptile != ent[i - 1].ptile) {
            if (new_row) rpb[ent[i].row] = npid;
            ++npid;
            rank[i] = 0;
        } else {
            rank[i] = rank[i - 1] + 1;
        }
        pid[i] = npid - 1;
        rpe[ent[i].row] = npid;
    }
    // producer side: entries grouped by tile (counting sort keeps the pid order)
    std::vector<int32_t> eptr(ntiles + 1, 0), qptr(ntiles + 1, 0), emeta(nent), qpid;
    std::vector<T> ew(nent);
    std::vector<int64_t> order(nent), tmp_order;
    for (int64_t i = 0; i < nent; ++i) eptr[ent[i].ptile + 1]++;
    for (int64_t tl = 0; tl < ntiles; ++tl) eptr[tl + 1] += eptr[tl];
    {
        std::vector<int32_t> fill(eptr.begin(), eptr.end() - 1);
        for (int64_t i = 0; i < nent; ++i) order[fill[ent[i].ptile]++] = i;
    }
    std::vector<int32_t> pos(nent), rcount;
    int max_q = 0;
    for (int64_t tl = 0; tl < ntiles; ++tl) {
        const int64_t i0 = eptr[tl], i1 = eptr[tl + 1];
        qptr[tl] = (int32_t)qpid.size();
        const int64_t q0 = (int64_t)qpid.size();
        int32_t maxr = 0;
        for (int64_t i = i0; i < i1; ++i) {
            if ((int64_t)qpid.size() == q0 || qpid.back() != pid[order[i]]) qpid.push_back(pid[order[i]]);
            pos[order[i]] = (int32_t)((int64_t)qpid.size() - 1 - q0);
            maxr = std::max(maxr, rank[order[i]]);
        }
        max_q = std::max(max_q, (int)((int64_t)qpid.size() - q0));
        // within the tile: by rank, then pid (a stable counting sort by rank of the
        // pid-ordered entries), so adjacent lanes add into different partial sums
        rcount.assign(maxr + 2, 0);
        for (int64_t i = i0; i < i1; ++i) rcount[rank[order[i]] + 1]++;
        for (int32_t r = 0; r <= maxr; ++r) rcount[r + 1] += rcount[r];
        tmp_order.resize(i1 - i0);
        for (int64_t i = i0; i < i1; ++i) tmp_order[rcount[rank[order[i]]]++] = order[i];
        for (int64_t k = i0; k < i1; ++k) {
            const int64_t e = tmp_order[k - i0];
            emeta[k] = (int32_t)((uint32_t)ent[e].field << 31 | (uint32_t)pos[e] << 11 | (uint32_t)ent[e].slot);
            ew[k] = (T)ent[e].w;
        }
    }
    qptr[ntiles] = (int32_t)qpid.size();
    if (max_q > STAG_MAXQ) {
        ib_set_error("a staggered step tile holds more correction partial sums than the kernel's buffer");
        return IB_ERR_STATE;
    }
    // consumer side: rows grouped by tile (counting sort)
    std::vector<int32_t> rptr(ntiles + 1, 0), rslot(nrow), rb(nrow), re(nrow);
    for (int64_t r = 0; r < nrow; ++r) rptr[rows[r].ctile + 1]++;
    for (int64_t tl = 0; tl < ntiles; ++tl) rptr[tl + 1] += rptr[tl];
    {
        std::vector<int32_t> fill(rptr.begin(), rptr.end() - 1);
        for (int64_t r = 0; r < nrow; ++r) {
            const int32_t i = fill[rows[r].ctile]++;
            rslot[i] = rows[r].cslot;
            rb[i] = rpb[r];
            re[i] = rpe[r];
        }
    }
    auto up = [&](auto** dst, const auto& v) -> ib_status {
        using E = typename std::decay<decltype(v[0])>::type;
        E* d;
        TRY(S.alloc(&d, (int64_t)std::max<size_t>(v.size(), 1)));
        if (!v.empty()) IB_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(E) * v.size(), cudaMemcpyHostToDevice, s));
        *dst = d;
        return IB_OK;
    };
    int32_t *d_eptr, *d_qptr, *d_qpid, *d_emeta, *d_rptr, *d_rslot, *d_rb, *d_re;
    T* d_ew;
    TRY(up(&d_eptr, eptr));
    TRY(up(&d_qptr, qptr));
    TRY(up(&d_qpid, qpid));
    TRY(up(&d_emeta, emeta));
    TRY(up(&d_ew, ew));
    TRY(up(&d_rptr, rptr));
    TRY(up(&d_rslot, rslot));
    TRY(up(&d_rb, rb));
    TRY(up(&d_re, re));
    T* partial;
    TRY(S.alloc(&partial, std::max<int64_t>(npid, 1), true));
    IB_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    prod.qptr = d_qptr;
    prod.qpid = d_qpid;
    prod.eptr = d_eptr;
    prod.emeta = d_emeta;
    prod.ew = d_ew;
    prod.out = partial;
    prod.max_q = max_q;
    cons.rptr = d_rptr;
    cons.rslot = d_rslot;
    cons.rpb = d_rb;
    cons.rpe = d_re;
    cons.in = partial;
    cons.n_in = npid;
    return IB_OK;
}

__global__ void k_add_step(int* base, int k) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *base += k;
}

// time steps per captured graph of the staggered loop (the graph is replayed nt / STAG_GRAPH_STEPS times)
static const int STAG_GRAPH_STEPS = 50;
static_assert(STAG_GRAPH_STEPS == STAB_BLOCK, "the stability probe renormalises between graph replays");

template <typename T>
static ib_status forward_stag(ib_table* t, const ib_shot* sh, double dt, int nt, cudaStream_t s,
                              const Probe* probe = nullptr) {
    const Layout& L = t->L;
    const int d = t->grid.ndim;
    if (shot_damped(sh)) {
        ib_set_error("the absorbing layer is implemented for the second-order form");
        return IB_ERR_STATE;
    }
    if (d != 2) {
        ib_set_error("the staggered form is implemented in 2D");
        return IB_ERR_STATE;
    }
    const int M = t->opts.space_order;
    const int H = M / 2;
    Scratch S(s);
    T *p, *vx, *vz, *kp, *bx, *bz;
    TRY(S.alloc(&p, L.total, true));
    TRY(S.alloc(&vx, L.total, true));
    TRY(S.alloc(&vz, L.total, true));
    TRY(S.alloc(&kp, L.total, true));
    TRY(S.alloc(&bx, L.total, true));
    TRY(S.alloc(&bz, L.total, true));
    k_stag_coef<T><<<grid1(L.N, 256), 256, 0, s>>>(L, (const T*)sh->vel_dev, (const T*)sh->rho_dev, t->mask_pad[0],
                                                   t->mask_pad[1], t->mask_pad[2], dt, 1.0 / t->grid.h, kp, bx, bz);
    IB_CHECK_LAUNCH("k_stag_coef");
    ib_count_launch("setup");
    if (probe) {   // random p, v_x, v_z on their interior nodes, normalised together
        k_rand_fill<T><<<grid1(L.total, 256), 256, 0, s>>>(L.total, kp, probe->seed, p, (T*)nullptr);
        k_rand_fill<T><<<grid1(L.total, 256), 256, 0, s>>>(L.total, bx, probe->seed + 1, vx, (T*)nullptr);
        k_rand_fill<T><<<grid1(L.total, 256), 256, 0, s>>>(L.total, bz, probe->seed + 2, vz, (T*)nullptr);
        IB_CHECK_LAUNCH("k_rand_fill");
        TRY(probe_rescale<T>(probe, 0, L.total, p, vx, vz, s));
    }
    Geom<T> g;
    TRY(setup_points<T>(t, sh, dt / pow(t->grid.h, d), S, g));
    StagArgs<T> a;
    memset(&a, 0, sizeof a);
    a.L = L;
    {
        T w2u[5];
        stencil_weights<T>(M, w2u, a.c1);
    }
    a.p = p;
    a.vx = vx;
    a.vz = vz;
    a.bx = bx;
    a.bz = bz;
    a.kp = kp;
    constexpr int TZ = StagTile<T>::TZ, STG = StagTile<T>::STG;
    // p rows read partials of v (formed by the v kernel); v rows read partials of p
    TRY(build_stag_plan<T>(t, {{2, 0, 0}, {3, 0, 1}}, TZ, S, a.pp, a.pv, s));
    TRY(build_stag_plan<T>(t, {{0, 0, 0}, {1, 1, 0}}, TZ, S, a.pv, a.pp, s));
    const int64_t ntx = (L.nx + STAG_TX - 1) / STAG_TX, ntz = (L.nz + TZ - 1) / TZ;
    {
        std::vector<uint8_t> flag(ntx * ntz, 0);
        std::vector<int64_t> hidx(8 * (size_t)g.src.n);
        if (g.src.n) IB_CUDA(cudaMemcpy(hidx.data(), g.src.idx, 8 * hidx.size(), cudaMemcpyDeviceToHost));
        for (int64_t q : hidx) {
            const int64_t rel = q - L.base, z = rel / L.px, x = rel - z * L.px;
            if (x >= 0 && x < L.nx && z >= 0 && z < L.nz) flag[(z / TZ) * ntx + x / STAG_TX] = 1;
        }
        uint8_t* d;
        TRY(S.alloc(&d, (int64_t)flag.size()));
        IB_CUDA(cudaMemcpyAsync(d, flag.data(), flag.size(), cudaMemcpyHostToDevice, s));
        IB_CUDA(cudaStreamSynchronize(s));
        a.src_tile = d;
    }
    a.src = g.src;
    a.wavelet = (const T*)sh->wavelet_dev;
    a.rec = g.rec;
    a.traces = (T*)sh->traces_dev;
    a.nt = nt;
    dim3 grid2((unsigned)ntx, (unsigned)ntz);
    auto launch_step = [&](cudaStream_t st, bool prof) -> ib_status {
        auto v = [&]() {
            if (H == 1) k_stag_v2d<T, 1, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
            else if (H == 2) k_stag_v2d<T, 2, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
            else if (H == 3) k_stag_v2d<T, 3, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
            else k_stag_v2d<T, 4, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
        };
        auto pk = [&]() {
            if (H == 1) k_stag_p2d<T, 1, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
            else if (H == 2) k_stag_p2d<T, 2, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
            else if (H == 3) k_stag_p2d<T, 3, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
            else k_stag_p2d<T, 4, STAG_TX, TZ, STAG_MAXQ, STG><<<grid2, 256, 0, st>>>(a);
        };
        if (prof) {
            PROF_LAUNCH(kname<T>("stag_v2d_f32", "stag_v2d_f64"), st, { v(); });
            PROF_LAUNCH(kname<T>("stag_p2d_f32", "stag_p2d_f64"), st, { pk(); });
        } else {
            v();
            pk();
            ib_count_launch(kname<T>("stag_v2d_f32", "stag_v2d_f64"));
            ib_count_launch(kname<T>("stag_p2d_f32", "stag_p2d_f64"));
        }
        IB_CHECK_LAUNCH("staggered step");
        return IB_OK;
    };
    int* d_base;
    TRY(S.alloc(&d_base, 1, true));
    a.step_base = d_base;
    const int K = STAG_GRAPH_STEPS;
    const int nrep = (nt >= 2 * K && !getenv("IB_NO_GRAPH")) ? nt / K : 0;
    cudaStream_t cs = s;
    cudaEvent_t ready = nullptr;
    if (nrep) {
        // K steps (and the step-offset bump) as one graph, replayed nrep times on a side stream
        IB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        IB_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        IB_CUDA(cudaEventRecord(ready, s));
        IB_CUDA(cudaStreamWaitEvent(cs, ready, 0));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        IB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        ib_status st = IB_OK;
        for (int k = 0; k < K && st == IB_OK; ++k) {
            a.step = k;
            a.rec_step = k - 1;
            st = launch_step(cs, false);
        }
        k_add_step<<<1, 32, 0, cs>>>(d_base, K);
        cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (st != IB_OK) return st;
        if (ce != cudaSuccess) return ib_cuda_fail(ce, "graph capture", __FILE__, __LINE__);
        IB_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        for (int r = 0; r < nrep; ++r) {
            ProfToken tk = ib_prof_begin(kname<T>("stag_graph50_f32", "stag_graph50_f64"), cs);
            IB_CUDA(cudaGraphLaunch(exec, cs));
            ib_prof_end(tk, cs);
            if (probe)
                TRY(probe_rescale<T>(probe, r + 1, L.total, p, vx, vz, cs, const_cast<T*>(a.pv.in), a.pv.n_in));
            for (int k = 0; k < K; ++k) {
                ib_count_launch(kname<T>("stag_v2d_f32", "stag_v2d_f64"));
                ib_count_launch(kname<T>("stag_p2d_f32", "stag_p2d_f64"));
            }
        }
        IB_CUDA(cudaStreamSynchronize(cs));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
    }
    for (int k = 0; k < nt - nrep * K; ++k) {     // the remaining steps, offset by the graphs' bumps
        a.step = k;
        a.rec_step = k - 1;
        TRY(launch_step(cs, true));
        if (probe && (nrep * K + k + 1) % STAB_BLOCK == 0)
            TRY(probe_rescale<T>(probe, (nrep * K + k + 1) / STAB_BLOCK, L.total, p, vx, vz, cs,
                                 const_cast<T*>(a.pv.in), a.pv.n_in));
    }
    if (g.rec.n) {
        k_receivers<T><<<grid1(g.rec.n, 256), 256, 0, cs>>>(g.rec, p, (T*)sh->traces_dev, nt, nt - 1);
        IB_CHECK_LAUNCH("k_receivers");
        ib_count_launch("setup");
    }
    if (!probe) TRY(check_finite<T>(L.total, p, vx, vz, cs));
    if (nrep) {
        IB_CUDA(cudaEventRecord(ready, cs));
        IB_CUDA(cudaStreamWaitEvent(s, ready, 0));
        IB_CUDA(cudaStreamSynchronize(cs));
        cudaEventDestroy(ready);
        cudaStreamDestroy(cs);
    }
    return IB_OK;
}

// ---------------------------------------------------------------------------
// 3D staggered pressure-velocity (1st-order section: the paper's signs and the
// backward-staggered base stencil; 3D first-order example), one thread per node:
//   v_a[j] (at j + e_a/2) += b_a[j] (sum_k c_k (p[j + k e_a] - p[j - (k-1) e_a]) + G_a corrections)
//   p[j] += kp[j] (sum_a sum_k c_k (v_a[j + (k-1) e_a] - v_a[j - k e_a]) + D corrections) + src
// with b_a = dt / (rho h) (mean of 1/rho at the two nodes) and kp = dt rho c^2 / h.
// The corrections of the modified rows follow each update in a pass over the
// rows of each operator (k_ib_rows, 8 lanes per row): the updated field is not
// read by its own update, so the pass sees the same values the fused sum would.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_stag_coef3(Layout L, const T* vel, const T* rho, const uint8_t* mp, const uint8_t* mv0,
                             const uint8_t* mv1, const uint8_t* mv2, double dt, double inv_h, T* kp, T* b0, T* b1,
                             T* b2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % L.nx, r = i / L.nx, y = r % L.ny, z = r / L.ny;
        const int64_t q = L.idx(x, y, z);
        const double r0 = rho ? (double)rho[i] : 1.0;
        const double c = (double)vel[i];
        kp[q] = mp[q] ? (T)(dt * r0 * c * c * inv_h) : (T)0;
        const double rx = (rho && x + 1 < L.nx) ? (double)rho[i + 1] : r0;
        const double ry = (rho && y + 1 < L.ny) ? (double)rho[i + L.nx] : r0;
        const double rz = (rho && z + 1 < L.nz) ? (double)rho[i + L.nx * L.ny] : r0;
        b0[q] = mv0[q] ? (T)(dt * 0.5 * (1.0 / r0 + 1.0 / rx) * inv_h) : (T)0;
        b1[q] = mv1[q] ? (T)(dt * 0.5 * (1.0 / r0 + 1.0 / ry) * inv_h) : (T)0;
        b2[q] = mv2[q] ? (T)(dt * 0.5 * (1.0 / r0 + 1.0 / rz) * inv_h) : (T)0;
    }
}

template <typename T, int H>
struct Stag3Args {
    Layout L;
    T c[4];              // c[k - 1]: weight of the pair at offsets +(k - 1/2), -(k - 1/2)
    T* p;
    T* v[3];
    const T* kp;
    const T* b[3];
};

// v_a += b_a (forward-staggered d/dx_a p) at every interior v_a node
template <typename T, int H>
__global__ void __launch_bounds__(256) k_stag_v3d(Stag3Args<T, H> a) {
    const Layout& L = a.L;
    const int64_t st[3] = {1, L.px, L.plane};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % L.nx, r = i / L.nx, y = r % L.ny, z = r / L.ny;
        const int64_t q = L.idx(x, y, z);
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const T bq = a.b[ax][q];
            if (bq == (T)0) continue;
            T s = 0;
#pragma unroll
            for (int k = 1; k <= H; ++k) s += a.c[k - 1] * (a.p[q + k * st[ax]] - a.p[q - (k - 1) * st[ax]]);
            a.v[ax][q] += bq * s;
        }
    }
}

// p += kp (backward-staggered divergence of v) at every interior p node
template <typename T, int H>
__global__ void __launch_bounds__(256) k_stag_p3d(Stag3Args<T, H> a) {
    const Layout& L = a.L;
    const int64_t st[3] = {1, L.px, L.plane};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % L.nx, r = i / L.nx, y = r % L.ny, z = r / L.ny;
        const int64_t q = L.idx(x, y, z);
        const T kq = a.kp[q];
        if (kq == (T)0) continue;
        T s = 0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
            for (int k = 1; k <= H; ++k)
                s += a.c[k - 1] * (a.v[ax][q + (k - 1) * st[ax]] - a.v[ax][q - k * st[ax]]);
        a.p[q] += kq * s;
    }
}

// out[q] += coef[q] sum_j w_j f[q + col_j] over the rows of one operator, 8 lanes per
// row (rows are distinct nodes within an operator; the sum is added by a reduction
// that returns nothing)
template <typename T>
__global__ void __launch_bounds__(256) k_ib_rows(int64_t nrows, const int64_t* __restrict__ row_pad,
                                                 const int64_t* __restrict__ row_ptr,
                                                 const int64_t* __restrict__ col_pad, const T* __restrict__ w,
                                                 const T* __restrict__ f, const T* __restrict__ coef, T* out) {
    const int lane = threadIdx.x & 31, gl = lane & 7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t rb = warp * 4; rb < nrows; rb += nwarp * 4) {
        const int64_t r = rb + (lane >> 3);
        const bool act = r < nrows;
        const int64_t q = act ? row_pad[r] : 0;
        const int64_t j1 = act ? row_ptr[r + 1] : 0;
        T v = 0;
        for (int64_t j = (act ? row_ptr[r] : 0) + gl; j < j1; j += 8) v += w[j] * f[q + col_pad[j]];
        v += __shfl_xor_sync(0xffffffffu, v, 4, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 2, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 1, 8);
        if (act && gl == 0) atomicAdd(&out[q], coef[q] * v);
    }
}

// sources: p[corner] += w * wavelet[n] (weights include dt / h^d)
template <typename T>
__global__ void k_add_sources(PointSet<T> src, const T* wavelet, int n, T* p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 8 * src.n && src.w[i] != (T)0) atomicAdd(&p[src.idx[i]], src.w[i] * wavelet[n]);
}

template <typename T, int H>
static ib_status stag3_steps(ib_table* t, const ib_shot* sh, int nt, Stag3Args<T, H>& a, const Geom<T>& g,
                             cudaStream_t s) {
    const Layout& L = a.L;
    const int gb = grid1(L.N, 256);
    for (int n = 0; n < nt; ++n) {
        PROF_LAUNCH(kname<T>("stag_v3d_f32", "stag_v3d_f64"), s, { k_stag_v3d<T, H><<<gb, 256, 0, s>>>(a); });
        for (int ax = 0; ax < 3; ++ax) {
            const IbOp& op = t->ops[ax];
            if (!op.nrows) continue;
            const T* w = sizeof(T) == 8 ? (const T*)op.w64 : (const T*)op.w32;
            PROF_LAUNCH(kname<T>("ib_rows3_f32", "ib_rows3_f64"), s, {
                k_ib_rows<T><<<grid1(op.nrows * 8, 256), 256, 0, s>>>(op.nrows, op.row_pad, op.row_ptr, op.col_pad,
                                                                       w, a.p, a.b[ax], a.v[ax]);
            });
        }
        PROF_LAUNCH(kname<T>("stag_p3d_f32", "stag_p3d_f64"), s, { k_stag_p3d<T, H><<<gb, 256, 0, s>>>(a); });
        for (int ax = 0; ax < 3; ++ax) {
            const IbOp& op = t->ops[3 + ax];
            if (!op.nrows) continue;
            const T* w = sizeof(T) == 8 ? (const T*)op.w64 : (const T*)op.w32;
            PROF_LAUNCH(kname<T>("ib_rows3_f32", "ib_rows3_f64"), s, {
                k_ib_rows<T><<<grid1(op.nrows * 8, 256), 256, 0, s>>>(op.nrows, op.row_pad, op.row_ptr, op.col_pad,
                                                                       w, a.v[ax], a.kp, a.p);
            });
        }
        if (g.src.n) {
            k_add_sources<T><<<1, 256, 0, s>>>(g.src, (const T*)sh->wavelet_dev, n, a.p);
            ib_count_launch("setup");
        }
        if (g.rec.n) {
            k_receivers<T><<<grid1(g.rec.n, 256), 256, 0, s>>>(g.rec, a.p, (T*)sh->traces_dev, nt, n);
            ib_count_launch("setup");
        }
        IB_CHECK_LAUNCH("3D staggered step");
    }
    return IB_OK;
}

template <typename T>
static ib_status forward_stag3(ib_table* t, const ib_shot* sh, double dt, int nt, cudaStream_t s) {
    const Layout& L = t->L;
    if (shot_damped(sh)) {
        ib_set_error("the absorbing layer is implemented for the second-order form");
        return IB_ERR_STATE;
    }
    const int M = t->opts.space_order;
    const int H = M / 2;
    Scratch S(s);
    T *p, *v0, *v1, *v2, *kp, *b0, *b1, *b2;
    TRY(S.alloc(&p, L.total, true));
    TRY(S.alloc(&v0, L.total, true));
    TRY(S.alloc(&v1, L.total, true));
    TRY(S.alloc(&v2, L.total, true));
    TRY(S.alloc(&kp, L.total, true));
    TRY(S.alloc(&b0, L.total, true));
    TRY(S.alloc(&b1, L.total, true));
    TRY(S.alloc(&b2, L.total, true));
    k_stag_coef3<T><<<grid1(L.N, 256), 256, 0, s>>>(L, (const T*)sh->vel_dev, (const T*)sh->rho_dev, t->mask_pad[0],
                                                    t->mask_pad[1], t->mask_pad[2], t->mask_pad[3], dt,
                                                    1.0 / t->grid.h, kp, b0, b1, b2);
    IB_CHECK_LAUNCH("k_stag_coef3");
    ib_count_launch("setup");
    Geom<T> g;
    TRY(setup_points<T>(t, sh, dt / pow(t->grid.h, 3), S, g));
    T w2u[5], c1[4];
    stencil_weights<T>(M, w2u, c1);
    auto run = [&](auto hc) -> ib_status {
        constexpr int HH = decltype(hc)::value;
        Stag3Args<T, HH> a;
        memset(&a, 0, sizeof a);
        a.L = L;
        for (int k = 0; k < 4; ++k) a.c[k] = c1[k];
        a.p = p;
        a.v[0] = v0;
        a.v[1] = v1;
        a.v[2] = v2;
        a.kp = kp;
        a.b[0] = b0;
        a.b[1] = b1;
        a.b[2] = b2;
        return stag3_steps<T, HH>(t, sh, nt, a, g, s);
    };
    if (H == 1) TRY(run(std::integral_constant<int, 1>()));
    else if (H == 2) TRY(run(std::integral_constant<int, 2>()));
    else if (H == 3) TRY(run(std::integral_constant<int, 3>()));
    else TRY(run(std::integral_constant<int, 4>()));
    TRY(check_finite<T>(L.total, p, v0, v1, s));
    TRY(check_finite<T>(L.total, v2, (const T*)nullptr, (const T*)nullptr, s));
    return IB_OK;
}

extern "C" ib_status ib_forward(const ib_table* tc, const ib_shot* sh, int32_t precision, double dt, int32_t nt,
                                void* ckpt, int32_t n_ckpt, void* stream) {
    ib_set_error("");
    TRY(check_shot(tc, sh, precision, dt, nt));
    ib_table* t = const_cast<ib_table*>(tc);
    cudaStream_t s = (cudaStream_t)stream;
    if (t->form == IB_SECOND_ORDER) {
        if (ckpt && n_ckpt < 1) {
            ib_set_error("n_ckpt must be >= 1");
            return IB_ERR_ARG;
        }
        return precision == 64 ? forward_2nd<double>(t, sh, dt, nt, ckpt, n_ckpt, s)
                               : forward_2nd<float>(t, sh, dt, nt, ckpt, n_ckpt, s);
    }
    if (ckpt) {
        ib_set_error("checkpoints are supported for the second-order form");
        return IB_ERR_STATE;
    }
    if (t->grid.ndim == 3)
        return precision == 64 ? forward_stag3<double>(t, sh, dt, nt, s) : forward_stag3<float>(t, sh, dt, nt, s);
    return precision == 64 ? forward_stag<double>(t, sh, dt, nt, s) : forward_stag<float>(t, sh, dt, nt, s);
}

// receiver injection rows: node -> (receiver, weight), regrouped on the host
template <typename T>
static ib_status build_injection(const Layout& L, const PointSet<T>& rec, Scratch& S, RowView<T>& view,
                                 std::vector<TileBins>& keep) {
    memset(&view, 0, sizeof view);
    if (rec.n == 0) return IB_OK;
    std::vector<int64_t> idx(8 * (size_t)rec.n);
    std::vector<T> w(8 * (size_t)rec.n);
    IB_CUDA(cudaMemcpyAsync(idx.data(), rec.idx, 8 * idx.size(), cudaMemcpyDeviceToHost, S.s));
    IB_CUDA(cudaMemcpyAsync(w.data(), rec.w, sizeof(T) * w.size(), cudaMemcpyDeviceToHost, S.s));
    IB_CUDA(cudaStreamSynchronize(S.s));
    struct E {
        int64_t q;
        int64_t r;
        T w;
    };
    std::vector<E> es;
    for (int r = 0; r < rec.n; ++r)
        for (int c = 0; c < 8; ++c)
            if (w[8 * r + c] != (T)0) es.push_back({idx[8 * r + c], r, w[8 * r + c]});
    std::sort(es.begin(), es.end(), [](const E& a, const E& b) { return a.q != b.q ? a.q < b.q : a.r < b.r; });
    std::vector<int64_t> rows, ptr, col;
    std::vector<T> ww;
    for (size_t i = 0; i < es.size(); ++i) {
        if (i == 0 || es[i].q != es[i - 1].q) {
            rows.push_back(es[i].q);
            ptr.push_back((int64_t)i);
        }
        col.push_back(es[i].r);
        ww.push_back(es[i].w);
    }
    ptr.push_back((int64_t)es.size());
    if (rows.empty()) return IB_OK;
    int64_t *drows, *dptr, *dcol;
    T* dw;
    TRY(S.alloc(&drows, (int64_t)rows.size()));
    TRY(S.alloc(&dptr, (int64_t)ptr.size()));
    TRY(S.alloc(&dcol, (int64_t)col.size()));
    TRY(S.alloc(&dw, (int64_t)ww.size()));
    IB_CUDA(cudaMemcpyAsync(drows, rows.data(), 8 * rows.size(), cudaMemcpyHostToDevice, S.s));
    IB_CUDA(cudaMemcpyAsync(dptr, ptr.data(), 8 * ptr.size(), cudaMemcpyHostToDevice, S.s));
    IB_CUDA(cudaMemcpyAsync(dcol, col.data(), 8 * col.size(), cudaMemcpyHostToDevice, S.s));
    IB_CUDA(cudaMemcpyAsync(dw, ww.data(), sizeof(T) * ww.size(), cudaMemcpyHostToDevice, S.s));
    TileBins b;
    TRY(ib_make_bins_ext(L, (int64_t)rows.size(), drows, TX2, 1, TZ2, b, S.s));
    keep.push_back(b);
    view.row_pad = drows;
    view.row_ptr = dptr;
    view.col = dcol;
    view.w = dw;
    view.tile_ptr = b.tile_ptr;
    view.perm = b.perm;
    view.ntx = b.ntx;
    IB_CUDA(cudaStreamSynchronize(S.s));
    return IB_OK;
}

template <typename T>
static ib_status adjoint_2nd(ib_table* t, const ib_shot* sh, double dt, int nt, const void* ckpt, int n_ckpt,
                             const T* res, T* grad_out, T* gw, cudaStream_t s) {
    const Layout& L = t->L;
    const int d = t->grid.ndim;
    if (d != 2) {
        ib_set_error("the adjoint is implemented in 2D");
        return IB_ERR_STATE;
    }
    const int M = t->opts.space_order;
    const int H = M / 2;
    Scratch S(s);
    T *Kh, *mu1, *mu2, *grad;
    TRY(S.alloc(&Kh, L.total, true));
    TRY(S.alloc(&mu1, L.total, true));
    TRY(S.alloc(&mu2, L.total, true));
    TRY(S.alloc(&grad, L.total, true));
    k_leap_coef<T><<<grid1(L.N, 256), 256, 0, s>>>(L, (const T*)sh->vel_dev, t->mask_pad[0], dt / t->grid.h, Kh);
    IB_CHECK_LAUNCH("k_leap_coef");
    ib_count_launch("setup");
    Geom<T> g;
    TRY(setup_points<T>(t, sh, dt * dt / pow(t->grid.h, d), S, g));
    const TileBins* fb = nullptr;
    const TileBins* tb = nullptr;
    TRY(ib_table_bins(t, 0, false, TX2, 1, TZ2, &fb, s));
    TRY(ib_table_bins(t, 0, true, TX2, 1, TZ2, &tb, s));
    std::vector<TileBins> keep;
    RowView<T> inj;
    TRY(build_injection<T>(L, g.rec, S, inj, keep));
    const int64_t seg = ckpt_seg(nt, n_ckpt);
    T* segbuf;
    TRY(S.alloc(&segbuf, (seg + 2) * L.total, true));
    if (gw) IB_CUDA(cudaMemsetAsync(gw, 0, sizeof(T) * nt, s));
    StepArgs<T> fa;
    memset(&fa, 0, sizeof fa);
    fa.L = L;
    {
        T c1u[4];
        stencil_weights<T>(M, fa.w2, c1u);
    }
    fa.Kh = Kh;
    fa.op = tview<T>(fb);
    fa.src = g.src;
    fa.wavelet = (const T*)sh->wavelet_dev;
    fa.rec.n = 0;
    fa.rec_step = -1;
    fa.nt = nt;
    set_damping<T>(sh, dt, fa.dw, fa.da);
    AdjArgs<T> aa;
    memset(&aa, 0, sizeof aa);
    aa.L = L;
    for (int k = 0; k < 5; ++k) aa.w2[k] = fa.w2[k];
    aa.Kh = Kh;
    aa.mask = t->mask_pad[0];
    aa.two_dt_over_h = (T)(2.0 * dt / t->grid.h);
    aa.opT = tview<T>(tb);
    aa.opT.ntx = (L.nx + TX2 - 1) / TX2;
    aa.inj = inj;
    aa.inj.ntx = aa.opT.ntx;
    aa.res = res;
    aa.nt = nt;
    aa.grad = grad;
    aa.src = g.src;
    aa.wavelet = (const T*)sh->wavelet_dev;
    aa.gw = gw;
    set_damping<T>(sh, dt, aa.dw, aa.da);
    dim3 grid2((unsigned)((L.nx + TX2 - 1) / TX2), (unsigned)((L.nz + TZ2 - 1) / TZ2));
    T* mu_a = mu1;   // mu^{m+1}
    T* mu_b = mu2;   // mu^{m+2}
    for (int k = n_ckpt - 1; k >= 0; --k) {
        const int64_t c = (int64_t)k * seg;
        if (c >= nt) continue;
        const int64_t e = std::min<int64_t>(c + seg, nt);
        const T* slot = (const T*)ckpt + (int64_t)k * 2 * L.total;
        // segment slots j hold p^{c - 1 + j}
        IB_CUDA(cudaMemcpyAsync(segbuf, slot + L.total, sizeof(T) * L.total, cudaMemcpyDeviceToDevice, s));
        IB_CUDA(cudaMemcpyAsync(segbuf + L.total, slot, sizeof(T) * L.total, cudaMemcpyDeviceToDevice, s));
        for (int64_t n = c; n < e; ++n) {
            fa.p = segbuf + (n - c + 1) * L.total;
            fa.pm = segbuf + (n - c) * L.total;
            fa.out = segbuf + (n - c + 2) * L.total;
            fa.step = (int)n;
            launch_leap2d<T>(fa, H, grid2, s);
            IB_CHECK_LAUNCH("recompute step");
        }
        for (int64_t m = e; m >= c + 1; --m) {
            aa.mu = mu_a;
            aa.mum = mu_b;
            aa.out = mu_b;
            aa.m = (int)m;
            aa.pm0 = segbuf + (m - c + 1) * L.total;
            aa.pm1 = segbuf + (m - c) * L.total;
            aa.pm2 = segbuf + (m - c - 1) * L.total;
            PROF_LAUNCH(kname<T>("adj2d_f32", "adj2d_f64"), s, {
                if (H == 1) k_adj2d<T, 1, TX2, TZ2><<<grid2, 256, 0, s>>>(aa);
                else if (H == 2) k_adj2d<T, 2, TX2, TZ2><<<grid2, 256, 0, s>>>(aa);
                else if (H == 3) k_adj2d<T, 3, TX2, TZ2><<<grid2, 256, 0, s>>>(aa);
                else k_adj2d<T, 4, TX2, TZ2><<<grid2, 256, 0, s>>>(aa);
            });
            IB_CHECK_LAUNCH("adjoint step");
            std::swap(mu_a, mu_b);
        }
    }
    k_unpad<T><<<grid1(L.N, 256), 256, 0, s>>>(L, grad, grad_out);
    IB_CHECK_LAUNCH("k_unpad");
    ib_count_launch("setup");
    TRY(check_finite<T>(L.N, grad_out, (const T*)nullptr, (const T*)nullptr, s));
    IB_CUDA(cudaStreamSynchronize(s));
    for (auto& b : keep) ib_free_bins(b);
    return IB_OK;
}

extern "C" ib_status ib_adjoint(const ib_table* tc, const ib_shot* sh, int32_t precision, double dt, int32_t nt,
                                const void* ckpt, int32_t n_ckpt, const void* residual, void* grad_vel,
                                void* grad_wavelet, void* stream) {
    ib_set_error("");
    TRY(check_shot(tc, sh, precision, dt, nt, false));
    if (!ckpt || n_ckpt < 1 || !residual || !grad_vel) {
        ib_set_error("adjoint needs checkpoints, residual and gradient buffers");
        return IB_ERR_ARG;
    }
    ib_table* t = const_cast<ib_table*>(tc);
    if (t->form != IB_SECOND_ORDER) {
        ib_set_error("the adjoint is implemented for the second-order form");
        return IB_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == 64)
        return adjoint_2nd<double>(t, sh, dt, nt, ckpt, n_ckpt, (const double*)residual, (double*)grad_vel,
                                   (double*)grad_wavelet, s);
    return adjoint_2nd<float>(t, sh, dt, nt, ckpt, n_ckpt, (const float*)residual, (float*)grad_vel,
                              (float*)grad_wavelet, s);
}

// ---------------------------------------------------------------------------
// batched shots: one launch per time step over the tiles of every shot,
// captured with all nt steps into one CUDA graph; the tile shape is chosen by
// timing the candidates on the batch itself (cached per shape class)
// ---------------------------------------------------------------------------
struct TileShape {
    int tx, tz, nsub;   // nsub > 1: z-marched strips of nsub tiles (k_leap2d_batch_m)
};
static const int kNumShapes = 10;
static const TileShape kShapes[kNumShapes] = {{64, 8, 1},  {32, 16, 1}, {128, 4, 1}, {64, 4, 1},
                                              {64, 8, 8},  {64, 8, 8},  {64, 8, 8},  {64, 8, 8},
                                              {64, 16, 4}, {64, 16, 4}};

template <int H, int TX, int TZ>
static void launch_batch(const StepArgs<float>* args, const int64_t* tile0, const int32_t* shot_of, int nshot,
                         int step, int64_t nblk,
                         cudaStream_t s) {
    k_leap2d_batch<float, H, TX, TZ><<<(unsigned)nblk, 256, 0, s>>>(args, tile0, shot_of, nshot, step);
}

template <int H, int NSUB, int D, int MINB>
static void launch_batch_m(const StepArgs<float>* args, const int64_t* tile0, const int32_t* shot_of, int nshot,
                           int step, int64_t nblk, cudaStream_t s) {
    k_leap2d_batch_m<H, NSUB, D, MINB><<<(unsigned)nblk, 256, 0, s>>>(args, tile0, shot_of, nshot, step);
}

template <int H, int NSUB, int D, int MINB>
static void launch_batch_m4(const StepArgs<float>* args, const int64_t* tile0, const int32_t* shot_of, int nshot,
                            int step, int64_t nblk, cudaStream_t s) {
    constexpr size_t sm = Strip4<H, NSUB, D>::FLOATS * sizeof(float);
    static const bool attr = (cudaFuncSetAttribute(k_leap2d_batch_m4<H, NSUB, D, MINB>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                              true);
    (void)attr;
    k_leap2d_batch_m4<H, NSUB, D, MINB><<<(unsigned)nblk, 256, sm, s>>>(args, tile0, shot_of, nshot, step);
}

template <int H>
static void launch_batch_shape(int si, const StepArgs<float>* args, const int64_t* tile0, const int32_t* shot_of,
                               int nshot, int step,
                               int64_t nblk, cudaStream_t s) {
    switch (si) {
        case 0: launch_batch<H, 64, 8>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 1: launch_batch<H, 32, 16>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 2: launch_batch<H, 128, 4>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 3: launch_batch<H, 64, 4>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 4: launch_batch_m<H, 8, 2, 4>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 5: launch_batch_m<H, 8, 3, 4>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 6: launch_batch_m<H, 8, 2, 5>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 7: launch_batch_m<H, 8, 3, 5>(args, tile0, shot_of, nshot, step, nblk, s); break;
        case 8: launch_batch_m4<H, 4, 2, 3>(args, tile0, shot_of, nshot, step, nblk, s); break;
        default: launch_batch_m4<H, 4, 3, 3>(args, tile0, shot_of, nshot, step, nblk, s); break;
    }
}

static void launch_batch_any(int H, int si, const StepArgs<float>* args, const int64_t* tile0, const int32_t* shot_of,
                             int nshot, int step,
                             int64_t nblk, cudaStream_t s) {
    PROF_LAUNCH("leap2d_batch_f32", s, {
        if (H == 1) launch_batch_shape<1>(si, args, tile0, shot_of, nshot, step, nblk, s);
        else if (H == 2) launch_batch_shape<2>(si, args, tile0, shot_of, nshot, step, nblk, s);
        else if (H == 3) launch_batch_shape<3>(si, args, tile0, shot_of, nshot, step, nblk, s);
        else launch_batch_shape<4>(si, args, tile0, shot_of, nshot, step, nblk, s);
    });
}

static std::mutex g_tune_mu;
static std::map<std::pair<int, int64_t>, int> g_tuned;   // (H, total points / 2^18) -> shape index

struct BatchSetup {
    std::vector<StepArgs<float>> args;
    std::vector<int64_t> tile0;
    StepArgs<float>* d_args = nullptr;
    int64_t* d_tile0 = nullptr;
    int32_t* d_shot_of = nullptr;   // shot of each block
    int64_t nblk = 0;
};

static ib_status batch_prepare(ib_table* const* ts, const ib_shot* shots, int nshot, int si, double dt, int nt,
                               const std::vector<float*>& buf0, const std::vector<float*>& buf1,
                               const std::vector<float*>& Kh, const std::vector<Geom<float>>& geo, Scratch& S,
                               BatchSetup& B) {
    const int tx = kShapes[si].tx, tz = kShapes[si].tz;
    B.args.assign(nshot, StepArgs<float>());
    B.tile0.assign(nshot + 1, 0);
    for (int i = 0; i < nshot; ++i) {
        ib_table* t = ts[i];
        const Layout& L = t->L;
        const TileBins* bins = nullptr;
        TRY(ib_table_bins(t, 0, false, tx, 1, tz, &bins, S.s));
        StepArgs<float>& a = B.args[i];
        memset(&a, 0, sizeof a);
        a.L = L;
        float c1u[4];
        stencil_weights<float>(t->opts.space_order, a.w2, c1u);
        a.Kh = Kh[i];
        a.op = tview<float>(bins);
        a.src = geo[i].src;
        a.wavelet = (const float*)shots[i].wavelet_dev;
        a.rec = geo[i].rec;
        a.traces = (float*)shots[i].traces_dev;
        a.nt = nt;
        a.buf0 = buf0[i];
        a.buf1 = buf1[i];
        set_damping<float>(&shots[i], dt, a.dw, a.da);
        a.ntx = (L.nx + tx - 1) / tx;
        const int nsub = kShapes[si].nsub;
        int64_t ntiles = a.ntx * ((((L.nz + tz - 1) / tz) + nsub - 1) / nsub);
        a.ntiles = ntiles;
        // receivers are recorded by the first blocks of the shot: make sure there are enough
        int64_t need = (shots[i].nrec + 255) / 256;
        B.tile0[i + 1] = B.tile0[i] + std::max(ntiles, need);
    }
    B.nblk = B.tile0[nshot];
    TRY(S.alloc(&B.d_args, nshot));
    TRY(S.alloc(&B.d_tile0, nshot + 1));
    IB_CUDA(cudaMemcpyAsync(B.d_args, B.args.data(), sizeof(StepArgs<float>) * nshot, cudaMemcpyHostToDevice, S.s));
    IB_CUDA(cudaMemcpyAsync(B.d_tile0, B.tile0.data(), 8 * (nshot + 1), cudaMemcpyHostToDevice, S.s));
    std::vector<int32_t> shot_of(B.nblk);
    for (int i = 0; i < nshot; ++i)
        for (int64_t b = B.tile0[i]; b < B.tile0[i + 1]; ++b) shot_of[b] = i;
    TRY(S.alloc(&B.d_shot_of, std::max<int64_t>(B.nblk, 1)));
    IB_CUDA(cudaMemcpyAsync(B.d_shot_of, shot_of.data(), 4 * B.nblk, cudaMemcpyHostToDevice, S.s));
    IB_CUDA(cudaStreamSynchronize(S.s));   // the host table goes out of scope
    return IB_OK;
}

static ib_status forward_batch_impl(const ib_table* const* tables, const ib_shot* shots, int32_t nshot,
                                    int32_t precision, double dt, int32_t nt, void* const* ckpts, int32_t n_ckpt,
                                    void* stream) {
    ib_set_error("");
    if (ckpts && n_ckpt < 1) {
        ib_set_error("n_ckpt must be >= 1");
        return IB_ERR_ARG;
    }
    if (!tables || !shots || nshot < 1) {
        ib_set_error("empty batch");
        return IB_ERR_ARG;
    }
    if (precision != 32) {
        ib_set_error("batched shots run in FP32");
        return IB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<ib_table*> ts(nshot);
    int H = -1;
    for (int i = 0; i < nshot; ++i) {
        TRY(check_shot(tables[i], &shots[i], precision, dt, nt));
        ts[i] = const_cast<ib_table*>(tables[i]);
        if (ts[i]->form != IB_SECOND_ORDER || ts[i]->grid.ndim != 2) {
            ib_set_error("batched shots: 2D second-order tables only");
            return IB_ERR_STATE;
        }
        int h = ts[i]->opts.space_order / 2;
        if (H >= 0 && h != H) {
            ib_set_error("batched shots must share the space order");
            return IB_ERR_ARG;
        }
        H = h;
    }
    Scratch S(s);
    std::vector<float*> b0(nshot), b1(nshot), Kh(nshot);
    std::vector<Geom<float>> geo(nshot);
    int64_t total = 0;
    for (int i = 0; i < nshot; ++i) {
        const Layout& L = ts[i]->L;
        TRY(S.alloc(&b0[i], L.total, true));
        TRY(S.alloc(&b1[i], L.total, true));
        TRY(S.alloc(&Kh[i], L.total, true));
        k_leap_coef<float><<<grid1(L.N, 256), 256, 0, s>>>(L, (const float*)shots[i].vel_dev, ts[i]->mask_pad[0],
                                                           dt / ts[i]->grid.h, Kh[i]);
        IB_CHECK_LAUNCH("k_leap_coef");
        ib_count_launch("setup");
        TRY(setup_points<float>(ts[i], &shots[i], dt * dt / pow(ts[i]->grid.h, 2), S, geo[i]));
        total += L.N;
    }
    // ---- tile-shape autotuning (first batch of a shape class); IB_BATCH_SHAPE=<index
    // into kShapes> fixes the shape instead
    int best = 0;
    const char* forced = getenv("IB_BATCH_SHAPE");
    if (forced && *forced) {
        best = atoi(forced);
        if (best < 0 || best >= kNumShapes) {
            ib_set_error("IB_BATCH_SHAPE must name a tile shape index in [0, 10)");
            return IB_ERR_ARG;
        }
    } else {
        std::pair<int, int64_t> key(H, total >> 18);
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                best = it->second;
                have = true;
            }
        }
        if (!have) {
            float best_ms = 1e30f;
            cudaEvent_t e0, e1;
            IB_CUDA(cudaEventCreate(&e0));
            IB_CUDA(cudaEventCreate(&e1));
            for (int si = 0; si < kNumShapes; ++si) {
                BatchSetup B;
                TRY(batch_prepare(ts.data(), shots, nshot, si, dt, nt, b0, b1, Kh, geo, S, B));
                const int trial = std::min(nt, 12);
                for (int n = 0; n < 2; ++n) launch_batch_any(H, si, B.d_args, B.d_tile0, B.d_shot_of, nshot, n, B.nblk, s);
                IB_CUDA(cudaEventRecord(e0, s));
                for (int n = 0; n < trial; ++n) launch_batch_any(H, si, B.d_args, B.d_tile0, B.d_shot_of, nshot, n, B.nblk, s);
                IB_CUDA(cudaEventRecord(e1, s));
                IB_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                IB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best = si;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = best;
            // trial steps wrote the wavefields: start the real run from zero
            for (int i = 0; i < nshot; ++i) {
                IB_CUDA(cudaMemsetAsync(b0[i], 0, sizeof(float) * ts[i]->L.total, s));
                IB_CUDA(cudaMemsetAsync(b1[i], 0, sizeof(float) * ts[i]->L.total, s));
            }
        }
    }
    BatchSetup B;
    TRY(batch_prepare(ts.data(), shots, nshot, best, dt, nt, b0, b1, Kh, geo, S, B));
    // checkpoint copies (ib_forward's layout: slot k = [p^{k seg}, p^{k seg - 1}])
    ShotCopy<float>* d_items = nullptr;
    int64_t seg = 0, maxtot = 0;
    if (ckpts) {
        std::vector<ShotCopy<float>> items(nshot);
        for (int i = 0; i < nshot; ++i) {
            if (!ckpts[i]) {
                ib_set_error("null checkpoint buffer");
                return IB_ERR_ARG;
            }
            items[i] = {b0[i], b1[i], (float*)ckpts[i], ts[i]->L.total};
            maxtot = std::max(maxtot, ts[i]->L.total);
        }
        TRY(S.alloc(&d_items, nshot));
        IB_CUDA(cudaMemcpyAsync(d_items, items.data(), sizeof(ShotCopy<float>) * nshot, cudaMemcpyHostToDevice, s));
        IB_CUDA(cudaStreamSynchronize(s));
        seg = ckpt_seg(nt, n_ckpt);
    }
    const dim3 cgrid((unsigned)std::min<int64_t>((maxtot + 255) / 256, 256), (unsigned)nshot);
    // ---- all nt steps as one captured graph
    cudaStream_t cs;
    IB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ready;
    IB_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    IB_CUDA(cudaEventRecord(ready, s));
    IB_CUDA(cudaStreamWaitEvent(cs, ready, 0));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    IB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int n = 0; n < nt; ++n) {
        if (d_items && n % seg == 0) k_ckpt_batch<float><<<cgrid, 256, 0, cs>>>(d_items, n, (int)(n / seg));
        StepArgs<float>* dargs = B.d_args;
        switch (H) {
            case 1: launch_batch_shape<1>(best, dargs, B.d_tile0, B.d_shot_of, nshot, n, B.nblk, cs); break;
            case 2: launch_batch_shape<2>(best, dargs, B.d_tile0, B.d_shot_of, nshot, n, B.nblk, cs); break;
            case 3: launch_batch_shape<3>(best, dargs, B.d_tile0, B.d_shot_of, nshot, n, B.nblk, cs); break;
            default: launch_batch_shape<4>(best, dargs, B.d_tile0, B.d_shot_of, nshot, n, B.nblk, cs); break;
        }
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ce != cudaSuccess) return ib_cuda_fail(ce, "graph capture", __FILE__, __LINE__);
    IB_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    {
        ProfToken tk = ib_prof_begin("leap2d_batch_graph_f32", cs);
        IB_CUDA(cudaGraphLaunch(exec, cs));
        ib_prof_end(tk, cs);
        for (int n = 0; n < nt; ++n) ib_count_launch("leap2d_batch_f32");
    }
    // final receivers per shot
    for (int i = 0; i < nshot; ++i) {
        if (!geo[i].rec.n) continue;
        float* cur = (nt & 1) ? b1[i] : b0[i];
        k_receivers<float><<<grid1(geo[i].rec.n, 256), 256, 0, cs>>>(geo[i].rec, cur, (float*)shots[i].traces_dev,
                                                                      nt, nt - 1);
        ib_count_launch("setup");
    }
    IB_CHECK_LAUNCH("k_receivers");
    for (int i = 0; i < nshot; ++i) TRY(check_finite<float>(ts[i]->L.total, b0[i], b1[i], (const float*)nullptr, cs));
    IB_CUDA(cudaEventRecord(ready, cs));
    IB_CUDA(cudaStreamWaitEvent(s, ready, 0));
    IB_CUDA(cudaStreamSynchronize(cs));
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaEventDestroy(ready);
    cudaStreamDestroy(cs);
    return IB_OK;
}

extern "C" ib_status ib_forward_batch(const ib_table* const* tables, const ib_shot* shots, int32_t nshot,
                                      int32_t precision, double dt, int32_t nt, void* stream) {
    return forward_batch_impl(tables, shots, nshot, precision, dt, nt, nullptr, 0, stream);
}

extern "C" ib_status ib_forward_batch_ckpt(const ib_table* const* tables, const ib_shot* shots, int32_t nshot,
                                           int32_t precision, double dt, int32_t nt, void* const* ckpts,
                                           int32_t n_ckpt, void* stream) {
    if (!ckpts) {
        ib_set_error("null checkpoint array");
        return IB_ERR_ARG;
    }
    return forward_batch_impl(tables, shots, nshot, precision, dt, nt, ckpts, n_ckpt, stream);
}

// ---------------------------------------------------------------------------
// batched adjoint: every shot's segments in lockstep, one graph for the whole
// backward pass (segment restore, batched recompute steps, batched adjoint steps)
// ---------------------------------------------------------------------------
// block maps: tile0 / shot_of over 64 x 8 tiles (adjoint steps), stile0 / sshot_of
// over z-marched strips (recompute steps)
template <int H>
static void launch_adj_batch_h(const StepArgs<float>* fargs, const AdjBatch<float>* aargs, const ShotCopy<float>* rst,
                               const int64_t* tile0, const int32_t* shot_of, int64_t nblk, const int64_t* stile0,
                               const int32_t* sshot_of, int64_t nsblk, dim3 cgrid, int nt, int64_t c, int64_t e,
                               int k, cudaStream_t s) {
    k_seg_restore_batch<float><<<cgrid, 256, 0, s>>>(rst, k);
    for (int64_t n = c; n < e; ++n)
        k_leap2d_batch_seg_m<H, STRIP_NSUB, STRIP_D><<<(unsigned)nsblk, 256, 0, s>>>(fargs, stile0, sshot_of, (int)n,
                                                                                      (int)(n - c));
    for (int64_t m = e; m >= c + 1; --m)
        k_adj2d_batch<float, H, 64, 8><<<(unsigned)nblk, 256, 0, s>>>(aargs, tile0, shot_of, (int)m, (int)(m - c), nt);
}

extern "C" ib_status ib_adjoint_batch(const ib_table* const* tables, const ib_shot* shots, int32_t nshot,
                                      int32_t precision, double dt, int32_t nt, const void* const* ckpts,
                                      int32_t n_ckpt, const void* const* residuals, void* const* grads,
                                      void* stream) {
    ib_set_error("");
    if (!tables || !shots || nshot < 1 || !ckpts || !residuals || !grads || n_ckpt < 1) {
        ib_set_error("batched adjoint needs tables, shots, checkpoints, residuals and gradients");
        return IB_ERR_ARG;
    }
    if (precision != 32) {
        ib_set_error("batched shots run in FP32");
        return IB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<ib_table*> ts(nshot);
    int H = -1;
    for (int i = 0; i < nshot; ++i) {
        TRY(check_shot(tables[i], &shots[i], precision, dt, nt, false));
        ts[i] = const_cast<ib_table*>(tables[i]);
        if (ts[i]->form != IB_SECOND_ORDER || ts[i]->grid.ndim != 2) {
            ib_set_error("batched adjoint: 2D second-order tables only");
            return IB_ERR_STATE;
        }
        if (!ckpts[i] || !residuals[i] || !grads[i]) {
            ib_set_error("null checkpoint, residual or gradient buffer");
            return IB_ERR_ARG;
        }
        const int h = ts[i]->opts.space_order / 2;
        if (H >= 0 && h != H) {
            ib_set_error("batched shots must share the space order");
            return IB_ERR_ARG;
        }
        H = h;
    }
    const int64_t seg = ckpt_seg(nt, n_ckpt);
    Scratch S(s);
    std::vector<StepArgs<float>> fargs(nshot);
    std::vector<AdjBatch<float>> aargs(nshot);
    std::vector<ShotCopy<float>> rst(nshot);
    std::vector<float*> grad(nshot);
    std::vector<int64_t> tile0(nshot + 1, 0), stile0(nshot + 1, 0);
    std::vector<TileBins> keep;
    int64_t maxtot = 0;
    for (int i = 0; i < nshot; ++i) {
        ib_table* t = ts[i];
        const Layout& L = t->L;
        float *Kh, *mu1, *mu2, *segbuf;
        TRY(S.alloc(&Kh, L.total, true));
        TRY(S.alloc(&mu1, L.total, true));
        TRY(S.alloc(&mu2, L.total, true));
        TRY(S.alloc(&grad[i], L.total, true));
        TRY(S.alloc(&segbuf, (seg + 2) * L.total, true));
        k_leap_coef<float><<<grid1(L.N, 256), 256, 0, s>>>(L, (const float*)shots[i].vel_dev, t->mask_pad[0],
                                                           dt / t->grid.h, Kh);
        IB_CHECK_LAUNCH("k_leap_coef");
        ib_count_launch("setup");
        Geom<float> g;
        TRY(setup_points<float>(t, &shots[i], dt * dt / pow(t->grid.h, 2), S, g));
        const TileBins* fb = nullptr;
        const TileBins* tb = nullptr;
        TRY(ib_table_bins(t, 0, false, TX2, 1, TZ2, &fb, s));
        TRY(ib_table_bins(t, 0, true, TX2, 1, TZ2, &tb, s));
        RowView<float> inj;
        TRY(build_injection<float>(L, g.rec, S, inj, keep));
        StepArgs<float>& fa = fargs[i];
        memset(&fa, 0, sizeof fa);
        fa.L = L;
        float c1u[4];
        stencil_weights<float>(t->opts.space_order, fa.w2, c1u);
        fa.Kh = Kh;
        fa.op = tview<float>(fb);
        fa.src = g.src;
        fa.wavelet = (const float*)shots[i].wavelet_dev;
        fa.rec.n = 0;
        fa.rec_step = -1;
        fa.nt = nt;
        set_damping<float>(&shots[i], dt, fa.dw, fa.da);
        fa.buf0 = segbuf;
        fa.ntx = (L.nx + TX2 - 1) / TX2;
        fa.ntiles = fa.ntx * ((L.nz + TZ2 - 1) / TZ2);
        AdjArgs<float>& aa = aargs[i].a;
        memset(&aa, 0, sizeof aa);
        aa.L = L;
        for (int k = 0; k < 5; ++k) aa.w2[k] = fa.w2[k];
        aa.Kh = Kh;
        aa.mask = t->mask_pad[0];
        aa.two_dt_over_h = (float)(2.0 * dt / t->grid.h);
        aa.opT = tview<float>(tb);
        aa.opT.ntx = fa.ntx;
        aa.inj = inj;
        aa.inj.ntx = fa.ntx;
        aa.res = (const float*)residuals[i];
        aa.nt = nt;
        aa.grad = grad[i];
        aa.src = g.src;
        aa.wavelet = (const float*)shots[i].wavelet_dev;
        aa.gw = nullptr;
        set_damping<float>(&shots[i], dt, aa.dw, aa.da);
        aargs[i].mu1 = mu1;
        aargs[i].mu2 = mu2;
        aargs[i].seg = segbuf;
        rst[i] = {(const float*)ckpts[i], nullptr, segbuf, L.total};
        tile0[i + 1] = tile0[i] + fa.ntiles;
        stile0[i + 1] = stile0[i] + fa.ntx * (((L.nz + TZ2 - 1) / TZ2 + STRIP_NSUB - 1) / STRIP_NSUB);
        maxtot = std::max(maxtot, L.total);
    }
    const int64_t nblk = tile0[nshot], nsblk = stile0[nshot];
    std::vector<int32_t> shot_of(nblk), sshot_of(nsblk);
    for (int i = 0; i < nshot; ++i) {
        for (int64_t b = tile0[i]; b < tile0[i + 1]; ++b) shot_of[b] = i;
        for (int64_t b = stile0[i]; b < stile0[i + 1]; ++b) sshot_of[b] = i;
    }
    StepArgs<float>* d_f;
    AdjBatch<float>* d_a;
    ShotCopy<float>* d_r;
    int64_t *d_t0, *d_st0;
    int32_t *d_so, *d_sso;
    TRY(S.alloc(&d_f, nshot));
    TRY(S.alloc(&d_a, nshot));
    TRY(S.alloc(&d_r, nshot));
    TRY(S.alloc(&d_t0, nshot + 1));
    TRY(S.alloc(&d_so, std::max<int64_t>(nblk, 1)));
    TRY(S.alloc(&d_st0, nshot + 1));
    TRY(S.alloc(&d_sso, std::max<int64_t>(nsblk, 1)));
    IB_CUDA(cudaMemcpyAsync(d_st0, stile0.data(), 8 * (nshot + 1), cudaMemcpyHostToDevice, s));
    IB_CUDA(cudaMemcpyAsync(d_sso, sshot_of.data(), 4 * nsblk, cudaMemcpyHostToDevice, s));
    IB_CUDA(cudaMemcpyAsync(d_f, fargs.data(), sizeof(StepArgs<float>) * nshot, cudaMemcpyHostToDevice, s));
    IB_CUDA(cudaMemcpyAsync(d_a, aargs.data(), sizeof(AdjBatch<float>) * nshot, cudaMemcpyHostToDevice, s));
    IB_CUDA(cudaMemcpyAsync(d_r, rst.data(), sizeof(ShotCopy<float>) * nshot, cudaMemcpyHostToDevice, s));
    IB_CUDA(cudaMemcpyAsync(d_t0, tile0.data(), 8 * (nshot + 1), cudaMemcpyHostToDevice, s));
    IB_CUDA(cudaMemcpyAsync(d_so, shot_of.data(), 4 * nblk, cudaMemcpyHostToDevice, s));
    IB_CUDA(cudaStreamSynchronize(s));   // the host tables go out of scope
    const dim3 cgrid((unsigned)std::min<int64_t>((maxtot + 255) / 256, 256), (unsigned)nshot);
    // ---- the whole backward pass as one captured graph
    cudaStream_t cs;
    IB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ready;
    IB_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    IB_CUDA(cudaEventRecord(ready, s));
    IB_CUDA(cudaStreamWaitEvent(cs, ready, 0));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    IB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int64_t nadj = 0;
    for (int k = n_ckpt - 1; k >= 0; --k) {
        const int64_t c = (int64_t)k * seg;
        if (c >= nt) continue;
        const int64_t e = std::min<int64_t>(c + seg, nt);
        switch (H) {
            case 1: launch_adj_batch_h<1>(d_f, d_a, d_r, d_t0, d_so, nblk, d_st0, d_sso, nsblk, cgrid, nt, c, e, k, cs); break;
            case 2: launch_adj_batch_h<2>(d_f, d_a, d_r, d_t0, d_so, nblk, d_st0, d_sso, nsblk, cgrid, nt, c, e, k, cs); break;
            case 3: launch_adj_batch_h<3>(d_f, d_a, d_r, d_t0, d_so, nblk, d_st0, d_sso, nsblk, cgrid, nt, c, e, k, cs); break;
            default: launch_adj_batch_h<4>(d_f, d_a, d_r, d_t0, d_so, nblk, d_st0, d_sso, nsblk, cgrid, nt, c, e, k, cs); break;
        }
        nadj += e - c;
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ce != cudaSuccess) return ib_cuda_fail(ce, "graph capture", __FILE__, __LINE__);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return ib_cuda_fail(ce, "graph instantiate", __FILE__, __LINE__);
    }
    {
        ProfToken tk = ib_prof_begin("adj2d_batch_graph_f32", cs);
        IB_CUDA(cudaGraphLaunch(exec, cs));
        ib_prof_end(tk, cs);
        for (int64_t q = 0; q < nadj; ++q) {
            ib_count_launch("adj2d_batch_f32");
            ib_count_launch("leap2d_batch_seg_f32");
        }
    }
    for (int i = 0; i < nshot; ++i) {
        const Layout& L = ts[i]->L;
        k_unpad<float><<<grid1(L.N, 256), 256, 0, cs>>>(L, grad[i], (float*)grads[i]);
        ib_count_launch("setup");
        TRY(check_finite<float>(L.N, (const float*)grads[i], (const float*)nullptr, (const float*)nullptr, cs));
    }
    IB_CHECK_LAUNCH("k_unpad");
    IB_CUDA(cudaEventRecord(ready, cs));
    IB_CUDA(cudaStreamWaitEvent(s, ready, 0));
    IB_CUDA(cudaStreamSynchronize(cs));
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaEventDestroy(ready);
    cudaStreamDestroy(cs);
    for (auto& b : keep) ib_free_bins(b);
    return IB_OK;
}

extern "C" ib_status ib_selftest_bounded_wait(void* stream) {
    ib_set_error("");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    int* err;
    TRY(S.alloc(&err, 1, true));
    k_wait_selftest<<<1, 32, 0, s>>>(err);
    IB_CHECK_LAUNCH("k_wait_selftest");
    int h = 0;
    IB_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    IB_CUDA(cudaStreamSynchronize(s));
    if (h) {
        ib_set_error("bounded device wait gave up (self-test: expected)");
        return IB_ERR_TIMEOUT;
    }
    return IB_OK;
}

extern "C" ib_status ib_sync_status(void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ib_cuda_fail(e, "stream", __FILE__, __LINE__);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ib_cuda_fail(e, "device", __FILE__, __LINE__);
    int word = 0;
    IB_CUDA(cudaMemcpyFromSymbolAsync(&word, g_dev_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    IB_CUDA(cudaStreamSynchronize(s));
    if (word) {
        const int zero = 0;
        IB_CUDA(cudaMemcpyToSymbolAsync(g_dev_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        IB_CUDA(cudaStreamSynchronize(s));
        ib_set_error("non-finite values (NaN/Inf) in the final wavefield or gradient of a run on this device: "
                     "the scheme is unstable for that model and time step");
        return IB_ERR_UNSTABLE;
    }
    return IB_OK;
}

extern "C" ib_status ib_stability(const ib_table* tc, const ib_shot* shot, int32_t precision, double dt,
                                  int32_t n_steps, uint64_t seed, double max_gain, double* growth, void* stream) {
    ib_set_error("");
    if (!tc || !shot || !shot->vel_dev || !growth || (precision != 32 && precision != 64) || !(dt > 0.0) ||
        n_steps < 1 || !(max_gain > 1.0)) {
        ib_set_error("ib_stability: table, shot with velocity and output required; precision 32 or 64, dt > 0, "
                     "n_steps >= 1, max_gain > 1");
        return IB_ERR_ARG;
    }
    ib_table* t = const_cast<ib_table*>(tc);
    if (t->form != IB_SECOND_ORDER && t->grid.ndim != 2) {
        ib_set_error("ib_stability: the staggered form is implemented in 2D");
        return IB_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // whole renormalisation blocks, an even number of them
    const int nblk = std::max(2, ((n_steps + STAB_BLOCK - 1) / STAB_BLOCK + 1) / 2 * 2);
    const int nt = nblk * STAB_BLOCK;
    Scratch S(s);
    Probe pr;
    pr.seed = seed;
    pr.nslot = nblk + 1;
    TRY(S.alloc(&pr.sums, pr.nslot, true));
    TRY(S.alloc(&pr.logs, pr.nslot, true));
    ib_shot sh;
    memset(&sh, 0, sizeof sh);
    sh.vel_dev = shot->vel_dev;
    sh.rho_dev = shot->rho_dev;
    sh.damp_eta = shot->damp_eta;
    sh.damp_width = shot->damp_width;
    TRY(check_shot(tc, &sh, precision, dt, n_steps));
    if (t->form == IB_SECOND_ORDER)
        TRY(precision == 64 ? forward_2nd<double>(t, &sh, dt, nt, nullptr, 0, s, &pr)
                            : forward_2nd<float>(t, &sh, dt, nt, nullptr, 0, s, &pr));
    else
        TRY(precision == 64 ? forward_stag<double>(t, &sh, dt, nt, s, &pr)
                            : forward_stag<float>(t, &sh, dt, nt, s, &pr));
    std::vector<double> logs(pr.nslot);
    IB_CUDA(cudaMemcpyAsync(logs.data(), pr.logs, sizeof(double) * pr.nslot, cudaMemcpyDeviceToHost, s));
    IB_CUDA(cudaStreamSynchronize(s));
    // per-step growth over the second half of the blocks (the first half lets the
    // dominant mode emerge from the random start)
    double acc = 0.0;
    for (int k = nblk / 2 + 1; k <= nblk; ++k) acc += logs[k];
    const double rate = acc / (double)((nblk - nblk / 2) * STAB_BLOCK);
    *growth = std::isfinite(rate) ? exp(rate) : INFINITY;
    if (!std::isfinite(rate) || rate * (double)n_steps > log(max_gain)) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "ib_stability: per-step growth %.6f amplifies an unstable mode by %.3g over %d steps "
                 "(limit %.3g)", *growth, std::isfinite(rate) ? exp(rate * (double)n_steps) : INFINITY, n_steps,
                 max_gain);
        ib_set_error(buf);
        return IB_ERR_UNSTABLE;
    }
    return IB_OK;
}

// ---------------------------------------------------------------------------
// ib_forward_noalloc: the 2D second-order FP32 forward with its scratch in a
// file-scope device array instead of stream-ordered allocations, for callers
// that may not allocate device memory (see include/ib.h).
// ---------------------------------------------------------------------------
#define IB_NOALLOC_SCRATCH_BYTES (64ll << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[IB_NOALLOC_SCRATCH_BYTES];

// one warp per IB row: out[q] += Kh[q] * sum_j w_j p[q + col_j]
__global__ void k_ib_rows_add(int64_t nrows, const int64_t* __restrict__ row_pad, const int64_t* __restrict__ row_ptr,
                              const int64_t* __restrict__ col_pad, const float* __restrict__ w,
                              const float* __restrict__ p, const float* __restrict__ Kh, float* out) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp; r < nrows; r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t q = row_pad[r];
        float s = 0.f;
        for (int64_t j = row_ptr[r] + lane; j < row_ptr[r + 1]; j += 32) s += w[j] * p[q + col_pad[j]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[q] += Kh[q] * s;
    }
}

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

// Device address of the static scratch for the current device.  Outside stream
// capture it is looked up on every call (a device reset or a new primary
// context reloads the module and can move the array); while `s` is capturing,
// the address remembered from the last uncaptured call on this device is used,
// so the first call on a device must come before any capture.
static ib_status noalloc_scratch(cudaStream_t s, unsigned char** out) {
    int dev = 0;
    IB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        ib_set_error("device index out of range for the static scratch");
        return IB_ERR_ARG;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    IB_CUDA(cudaStreamIsCapturing(s, &cap));
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return ib_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        g_noalloc_ptr[dev] = ptr;
    } else if (!g_noalloc_ptr[dev]) {
        ib_set_error("ib_forward_noalloc: the first call on a device must not be captured");
        return IB_ERR_STATE;
    }
    *out = (unsigned char*)g_noalloc_ptr[dev];
    return IB_OK;
}

static int64_t align256(int64_t b) { return (b + 255) & ~(int64_t)255; }

extern "C" ib_status ib_forward_noalloc(const ib_table* tc, const ib_shot* sh, double dt, int32_t nt, void* stream) {
    ib_set_error("");
    TRY(check_shot(tc, sh, 32, dt, nt));
    ib_table* t = const_cast<ib_table*>(tc);
    if (t->form != IB_SECOND_ORDER || t->grid.ndim != 2) {
        ib_set_error("ib_forward_noalloc: 2D second-order tables only");
        return IB_ERR_STATE;
    }
    if (shot_damped(sh)) {
        ib_set_error("ib_forward_noalloc: no absorbing layer");
        return IB_ERR_STATE;
    }
    const Layout& L = t->L;
    const int64_t field = align256(sizeof(float) * L.total);
    const int64_t srcb = align256(8 * (int64_t)sh->nsrc * (8 + 4));
    const int64_t recb = align256(8 * (int64_t)sh->nrec * (8 + 4));
    const int64_t need = 3 * field + 2 * srcb + 2 * recb + 4 * 256;
    if (need > IB_NOALLOC_SCRATCH_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf, "ib_forward_noalloc: needs %lld bytes of scratch, the static limit is %lld",
                 (long long)need, (long long)IB_NOALLOC_SCRATCH_BYTES);
        ib_set_error(buf);
        return IB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    TRY(noalloc_scratch(s, &base));
    int64_t off = 0;
    auto carve = [&](int64_t bytes) {
        unsigned char* p = base + off;
        off += align256(bytes);
        return p;
    };
    float* p0 = (float*)carve(sizeof(float) * L.total);
    float* p1 = (float*)carve(sizeof(float) * L.total);
    float* Kh = (float*)carve(sizeof(float) * L.total);
    int64_t* si = (int64_t*)carve(8 * 8 * (int64_t)std::max(sh->nsrc, 1));
    float* sw = (float*)carve(4 * 8 * (int64_t)std::max(sh->nsrc, 1));
    int64_t* ri = (int64_t*)carve(8 * 8 * (int64_t)std::max(sh->nrec, 1));
    float* rw = (float*)carve(4 * 8 * (int64_t)std::max(sh->nrec, 1));
    // every call starts from zero wavefields and a zero padding ring
    IB_CUDA(cudaMemsetAsync(p0, 0, sizeof(float) * L.total, s));
    IB_CUDA(cudaMemsetAsync(p1, 0, sizeof(float) * L.total, s));
    IB_CUDA(cudaMemsetAsync(Kh, 0, sizeof(float) * L.total, s));
    k_leap_coef<float><<<grid1(L.N, 256), 256, 0, s>>>(L, (const float*)sh->vel_dev, t->mask_pad[0], dt / t->grid.h,
                                                       Kh);
    if (sh->nsrc)
        k_interp_setup<float><<<grid1(sh->nsrc, 64), 64, 0, s>>>(sh->nsrc, sh->src_dev, 2, 1.0 / t->grid.h, L,
                                                                  t->mask_pad[0], dt * dt / (t->grid.h * t->grid.h),
                                                                  si, sw);
    if (sh->nrec)
        k_interp_setup<float><<<grid1(sh->nrec, 64), 64, 0, s>>>(sh->nrec, sh->rec_dev, 2, 1.0 / t->grid.h, L,
                                                                  t->mask_pad[0], 1.0, ri, rw);
    IB_CHECK_LAUNCH("ib_forward_noalloc setup");
    const int M = t->opts.space_order;
    const int H = M / 2;
    StepArgs<float> a;
    memset(&a, 0, sizeof a);
    a.L = L;
    {
        float c1u[4];
        stencil_weights<float>(M, a.w2, c1u);
    }
    a.Kh = Kh;
    a.src = {sh->nsrc, si, sw};
    a.wavelet = (const float*)sh->wavelet_dev;
    a.rec = {sh->nrec, ri, rw};
    a.traces = (float*)sh->traces_dev;
    a.nt = nt;
    const IbOp& op = t->ops[0];
    dim3 grid2((unsigned)((L.nx + TX2 - 1) / TX2), (unsigned)((L.nz + TZ2 - 1) / TZ2));
    float* cur = p0;
    float* prev = p1;
    for (int n = 0; n < nt; ++n) {
        a.p = cur;
        a.pm = prev;
        a.out = prev;
        a.step = n;
        a.rec_step = n - 1;
        if (H == 1) k_leap2d<float, 1, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
        else if (H == 2) k_leap2d<float, 2, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
        else if (H == 3) k_leap2d<float, 3, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
        else k_leap2d<float, 4, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
        if (op.nrows)
            k_ib_rows_add<<<grid1(op.nrows * 32, 256), 256, 0, s>>>(op.nrows, op.row_pad, op.row_ptr, op.col_pad,
                                                                     op.w32, cur, Kh, prev);
        IB_CHECK_LAUNCH("ib_forward_noalloc step");
        std::swap(cur, prev);
    }
    if (sh->nrec)
        k_receivers<float><<<grid1(sh->nrec, 256), 256, 0, s>>>(a.rec, cur, (float*)sh->traces_dev, nt, nt - 1);
    IB_CHECK_LAUNCH("ib_forward_noalloc receivers");
    return IB_OK;
}
