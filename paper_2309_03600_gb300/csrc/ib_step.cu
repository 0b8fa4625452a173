// Time stepping: fused leapfrog (2D, 3D), staggered pressure-velocity (2D),
// source injection, receiver interpolation, the exact discrete adjoint and
// checkpointed velocity gradients.
//
// Paper: p^{t+1} = 2p^t - p^{t-1} + dt^2 c^2 lap p + dt^2 f (2nd-order
// application section), first-order system with the paper's signs and a
// backward-staggered base stencil (1st-order section), modified operators near
// the boundary ("Reconciliation with the Interior Numerical Discretization"),
// zero Dirichlet outer edges (Examples section).
//
// Every step kernel works on a tile of outputs: the bulk stencil reads a
// shared-memory copy of the tile and its halo; the immersed-boundary rows that
// fall in the tile are then added by a warp-cooperative gather over the
// correction table (one warp per row, lanes over the row's entries); finally
// the update, source injection and masking are applied and the tile is written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
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

// correction table of one operator as seen by a step kernel
template <typename T>
struct OpView {
    const int64_t* row_pad;
    const int64_t* row_ptr;
    const int64_t* col_pad;
    const T* w;
    const int32_t* tile_ptr;
    const int32_t* perm;
    int64_t ntx, nty;
};

template <typename T>
struct PointSet {                 // multilinear weights: 8 corner slots per point
    int n;
    const int64_t* idx;           // padded node
    const T* w;
};

template <typename T>
struct StepArgs {
    Layout L;
    T w2[5];             // central 2nd-derivative weights w[0..H]
    const T* p;          // current field p^n
    const T* pm;         // previous field p^{n-1}
    T* out;              // p^{n+1} (may alias pm)
    const T* K;          // dt^2 c^2 (0 outside the domain)
    T inv_h2;
    OpView<T> op;
    PointSet<T> src;     // weights include dt^2 / h^d
    const T* wavelet;
    int step;
    PointSet<T> rec;     // receivers sampled from p (the previous step's output)
    T* traces;
    int nt;
    int rec_step;        // trace column written from p (-1: none)
};

template <typename T>
__device__ __forceinline__ void record_receivers(const PointSet<T>& rec, const T* p, T* traces, int nt, int col) {
    int gid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    gid = gid * (blockDim.x * blockDim.y) + threadIdx.y * blockDim.x + threadIdx.x;
    if (col >= 0 && gid < rec.n) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) s += rec.w[8 * gid + c] * p[rec.idx[8 * gid + c]];
        traces[(int64_t)gid * nt + col] = s;
    }
}

// one warp per IB row of the tile: acc[local] += sum_k w_k f[row + col_k]
template <typename T, int TXA>
__device__ __forceinline__ void gather_rows(const OpView<T>& op, int64_t tile, const T* f, const Layout& L, int64_t x0,
                                            int64_t y0, T* acc, int accy) {
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    const int32_t b = op.tile_ptr[tile], e = op.tile_ptr[tile + 1];
    for (int k = b + warp; k < e; k += nw) {
        const int32_t r = op.perm[k];
        const int64_t q = op.row_pad[r];
        T s = 0;
        for (int64_t j = op.row_ptr[r] + lane; j < op.row_ptr[r + 1]; j += 32) s += op.w[j] * f[q + op.col_pad[j]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            int64_t loc = q - L.base;
            int64_t z = loc / L.plane;
            int64_t rem = loc - z * L.plane;
            int64_t y = rem / L.px;
            int64_t x = rem - y * L.px;
            if (L.ndim == 2) y = z;   // 2D: tile rows are z
            acc[(y - y0) * TXA + (x - x0)] += s;
        }
    }
    (void)accy;
}

// ---------------------------------------------------------------------------
// 2D leapfrog: tile TX x TZ, 256 threads (TX/32 outputs per thread per row)
// ---------------------------------------------------------------------------
template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256) k_leap2d(StepArgs<T> a) {
    __shared__ T tile[TZ + 2 * H][TX + 2 * H];
    __shared__ T acc[TZ * TX];
    const int tid = threadIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step);
    const int64_t x0 = (int64_t)blockIdx.x * TX, z0 = (int64_t)blockIdx.y * TZ;
    const Layout& L = a.L;
    for (int i = tid; i < (TZ + 2 * H) * (TX + 2 * H); i += 256) {
        int lz = i / (TX + 2 * H), lx = i - lz * (TX + 2 * H);
        int64_t x = x0 + lx - H, z = z0 + lz - H;
        T v = 0;
        if (x < L.nx + H && z < L.nz + H) v = a.p[L.base + z * L.px + x];
        tile[lz][lx] = v;
    }
    __syncthreads();
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        T c = tile[lz + H][lx + H];
        T s = (T)2 * a.w2[0] * c;
#pragma unroll
        for (int k = 1; k <= H; ++k)
            s += a.w2[k] * ((tile[lz + H][lx + H + k] + tile[lz + H][lx + H - k]) +
                             (tile[lz + H + k][lx + H] + tile[lz + H - k][lx + H]));
        acc[i] = s;
    }
    __syncthreads();
    if (a.op.tile_ptr) gather_rows<T, TX>(a.op, (int64_t)blockIdx.y * a.op.ntx + blockIdx.x, a.p, L, x0, z0, acc, TZ);
    __syncthreads();
    const T wv = a.src.n ? a.wavelet[a.step] : (T)0;
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        int64_t x = x0 + lx, z = z0 + lz;
        if (x >= L.nx || z >= L.nz) continue;
        int64_t q = L.base + z * L.px + x;
        T v = (T)2 * tile[lz + H][lx + H] - a.pm[q] + a.K[q] * (acc[i] * a.inv_h2);
        for (int s = 0; s < 8 * a.src.n; ++s)
            if (a.src.idx[s] == q) v += a.src.w[s] * wv;
        a.out[q] = v;
    }
}

// receivers only (after the last step)
template <typename T>
__global__ void k_receivers(PointSet<T> rec, const T* p, T* traces, int nt, int col) {
    record_receivers(rec, p, traces, nt, col);
}

// ---------------------------------------------------------------------------
// 3D leapfrog: (x, y) tile of 32 x 8 columns marching in z with a register
// queue of the 2H + 1 values of its own column; x/y neighbours from a
// shared-memory copy of the current plane with its halo.
// ---------------------------------------------------------------------------
template <typename T, int H>
__global__ void __launch_bounds__(256) k_leap3d(StepArgs<T> a, int zchunk) {
    constexpr int TX = 32, TY = 8;
    __shared__ T tile[TY + 2 * H][TX + 2 * H];
    __shared__ T acc[TY * TX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step);
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
        __syncthreads();
        {
            T s = (T)3 * a.w2[0] * q[H];
#pragma unroll
            for (int k = 1; k <= H; ++k)
                s += a.w2[k] * ((tile[ty + H][tx + H + k] + tile[ty + H][tx + H - k]) +
                                 (tile[ty + H + k][tx + H] + tile[ty + H - k][tx + H]) + (q[H + k] + q[H - k]));
            acc[tid] = s;
        }
        __syncthreads();
        if (a.op.tile_ptr)
            gather_rows<T, TX>(a.op, (z * a.op.nty + blockIdx.y) * a.op.ntx + blockIdx.x, a.p, L, x0, y0, acc, TY);
        __syncthreads();
        if (valid) {
            int64_t qi = L.idx(x, y, z);
            T v = (T)2 * q[H] - a.pm[qi] + a.K[qi] * (acc[tid] * a.inv_h2);
            for (int s = 0; s < 8 * a.src.n; ++s)
                if (a.src.idx[s] == qi) v += a.src.w[s] * wv;
            a.out[qi] = v;
        }
#pragma unroll
        for (int k = 0; k < 2 * H; ++k) q[k] = q[k + 1];
        // plane z + 1 + H exists only while z + 1 < ze (the last allocated plane is nz + H - 1)
        q[2 * H] = (col_ok && z + 1 < ze) ? a.p[L.idx(x, y, z + 1 + H)] : (T)0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 2D staggered pressure-velocity
//   v_a[j] (at j + e_a/2) += b_a[j] (sum_k c_k (p[j + k e_a] - p[j - (k-1) e_a]) + IB) / h
//   p[j] += kp[j] (sum_a sum_k c_k (v_a[j + (k-1) e_a] - v_a[j - k e_a]) + IB) / h + src
// ---------------------------------------------------------------------------
template <typename T>
struct StagArgs {
    Layout L;
    T c1[4];             // staggered weights for offsets +1/2 .. +(M-1)/2
    T* p;
    T* vx;
    T* vz;
    const T* bx;      // dt / rho at v_x nodes (0 outside)
    const T* bz;
    const T* kp;      // dt rho c^2 at p nodes (0 outside)
    T inv_h;
    OpView<T> gx, gz, dx, dz;
    PointSet<T> src;  // weights include dt / h^d
    const T* wavelet;
    int step;
    PointSet<T> rec;
    T* traces;
    int nt;
    int rec_step;
};

template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256) k_stag_v2d(StagArgs<T> a) {
    __shared__ T tile[TZ + 2 * H][TX + 2 * H];
    __shared__ T ax[TZ * TX];
    __shared__ T az[TZ * TX];
    const int tid = threadIdx.x;
    record_receivers(a.rec, a.p, a.traces, a.nt, a.rec_step);
    const int64_t x0 = (int64_t)blockIdx.x * TX, z0 = (int64_t)blockIdx.y * TZ;
    const Layout& L = a.L;
    for (int i = tid; i < (TZ + 2 * H) * (TX + 2 * H); i += 256) {
        int lz = i / (TX + 2 * H), lx = i - lz * (TX + 2 * H);
        int64_t x = x0 + lx - H, z = z0 + lz - H;
        T v = 0;
        if (x < L.nx + H && z < L.nz + H) v = a.p[L.base + z * L.px + x];
        tile[lz][lx] = v;
    }
    __syncthreads();
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        T sx = 0, sz = 0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            sx += a.c1[k - 1] * (tile[lz + H][lx + H + k] - tile[lz + H][lx + H - k + 1]);
            sz += a.c1[k - 1] * (tile[lz + H + k][lx + H] - tile[lz + H - k + 1][lx + H]);
        }
        ax[i] = sx;
        az[i] = sz;
    }
    __syncthreads();
    const int64_t tile_id = (int64_t)blockIdx.y * a.gx.ntx + blockIdx.x;
    if (a.gx.tile_ptr) gather_rows<T, TX>(a.gx, tile_id, a.p, L, x0, z0, ax, TZ);
    if (a.gz.tile_ptr) gather_rows<T, TX>(a.gz, tile_id, a.p, L, x0, z0, az, TZ);
    __syncthreads();
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        int64_t x = x0 + lx, z = z0 + lz;
        if (x >= L.nx || z >= L.nz) continue;
        int64_t q = L.base + z * L.px + x;
        a.vx[q] += a.bx[q] * (ax[i] * a.inv_h);
        a.vz[q] += a.bz[q] * (az[i] * a.inv_h);
    }
}

template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256) k_stag_p2d(StagArgs<T> a) {
    __shared__ T tvx[TZ][TX + 2 * H];
    __shared__ T tvz[TZ + 2 * H][TX];
    __shared__ T acc[TZ * TX];
    const int tid = threadIdx.x;
    const int64_t x0 = (int64_t)blockIdx.x * TX, z0 = (int64_t)blockIdx.y * TZ;
    const Layout& L = a.L;
    for (int i = tid; i < TZ * (TX + 2 * H); i += 256) {
        int lz = i / (TX + 2 * H), lx = i - lz * (TX + 2 * H);
        int64_t x = x0 + lx - H, z = z0 + lz;
        T v = 0;
        if (x < L.nx + H && z < L.nz + H) v = a.vx[L.base + z * L.px + x];
        tvx[lz][lx] = v;
    }
    for (int i = tid; i < (TZ + 2 * H) * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        int64_t x = x0 + lx, z = z0 + lz - H;
        T v = 0;
        if (x < L.nx + H && z < L.nz + H) v = a.vz[L.base + z * L.px + x];
        tvz[lz][lx] = v;
    }
    __syncthreads();
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        T s = 0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            s += a.c1[k - 1] * (tvx[lz][lx + H + k - 1] - tvx[lz][lx + H - k]);
            s += a.c1[k - 1] * (tvz[lz + H + k - 1][lx] - tvz[lz + H - k][lx]);
        }
        acc[i] = s;
    }
    __syncthreads();
    const int64_t tile_id = (int64_t)blockIdx.y * a.dx.ntx + blockIdx.x;
    if (a.dx.tile_ptr) gather_rows<T, TX>(a.dx, tile_id, a.vx, L, x0, z0, acc, TZ);
    __syncthreads();
    if (a.dz.tile_ptr) gather_rows<T, TX>(a.dz, tile_id, a.vz, L, x0, z0, acc, TZ);
    __syncthreads();
    const T wv = a.src.n ? a.wavelet[a.step] : (T)0;
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        int64_t x = x0 + lx, z = z0 + lz;
        if (x >= L.nx || z >= L.nz) continue;
        int64_t q = L.base + z * L.px + x;
        T v = a.p[q] + a.kp[q] * (acc[i] * a.inv_h);
        for (int s = 0; s < 8 * a.src.n; ++s)
            if (a.src.idx[s] == q) v += a.src.w[s] * wv;
        a.p[q] = v;
    }
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
    const T* K;
    const uint8_t* mask;
    T inv_h2;
    T dt;
    OpView<T> opT;       // transposed corrections (rows keyed by column node)
    OpView<T> inj;       // receiver injection rows: w = interpolation weight, col_pad = receiver id
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
};

template <typename T, int H, int TX, int TZ>
__global__ void __launch_bounds__(256) k_adj2d(AdjArgs<T> a) {
    __shared__ T tile[TZ + 2 * H][TX + 2 * H];
    __shared__ T acc[TZ * TX];
    const int tid = threadIdx.x;
    const int64_t x0 = (int64_t)blockIdx.x * TX, z0 = (int64_t)blockIdx.y * TZ;
    const Layout& L = a.L;
    for (int i = tid; i < (TZ + 2 * H) * (TX + 2 * H); i += 256) {
        int lz = i / (TX + 2 * H), lx = i - lz * (TX + 2 * H);
        int64_t x = x0 + lx - H, z = z0 + lz - H;
        T v = 0;
        if (x < L.nx + H && z < L.nz + H) {
            int64_t q = L.base + z * L.px + x;
            v = a.K[q] * a.mu[q];
        }
        tile[lz][lx] = v;
    }
    __syncthreads();
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        T c = tile[lz + H][lx + H];
        T s = (T)2 * a.w2[0] * c;
#pragma unroll
        for (int k = 1; k <= H; ++k)
            s += a.w2[k] * ((tile[lz + H][lx + H + k] + tile[lz + H][lx + H - k]) +
                             (tile[lz + H + k][lx + H] + tile[lz + H - k][lx + H]));
        acc[i] = s * a.inv_h2;
    }
    __syncthreads();
    const int64_t tile_id = (int64_t)blockIdx.y * a.opT.ntx + blockIdx.x;
    // transposed IB corrections: sum_i w_ij K_i mu_i
    if (a.opT.tile_ptr) {
        const int warp = tid >> 5, lane = tid & 31;
        for (int k = a.opT.tile_ptr[tile_id] + warp; k < a.opT.tile_ptr[tile_id + 1]; k += 8) {
            const int32_t r = a.opT.perm[k];
            const int64_t q = a.opT.row_pad[r];
            T s = 0;
            for (int64_t j = a.opT.row_ptr[r] + lane; j < a.opT.row_ptr[r + 1]; j += 32) {
                int64_t src = q + a.opT.col_pad[j];
                s += a.opT.w[j] * (a.K[src] * a.mu[src]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                int64_t loc = q - L.base;
                int64_t z = loc / L.px, x = loc - z * L.px;
                acc[(z - z0) * TX + (x - x0)] += s * a.inv_h2;
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        int64_t x = x0 + lx, z = z0 + lz;
        if (x >= L.nx || z >= L.nz) continue;
        int64_t q = L.base + z * L.px + x;
        acc[i] = a.mask[q] ? acc[i] : (T)0;
    }
    __syncthreads();
    // receiver residual injection R^T res^{m-1}
    if (a.inj.tile_ptr) {
        const int warp = tid >> 5, lane = tid & 31;
        for (int k = a.inj.tile_ptr[tile_id] + warp; k < a.inj.tile_ptr[tile_id + 1]; k += 8) {
            const int32_t r = a.inj.perm[k];
            const int64_t q = a.inj.row_pad[r];
            T s = 0;
            for (int64_t j = a.inj.row_ptr[r] + lane; j < a.inj.row_ptr[r + 1]; j += 32)
                s += a.inj.w[j] * a.res[a.inj.col_pad[j] * (int64_t)a.nt + (a.m - 1)];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                int64_t loc = q - L.base;
                int64_t z = loc / L.px, x = loc - z * L.px;
                acc[(z - z0) * TX + (x - x0)] += s;
            }
        }
    }
    __syncthreads();
    const T wv = a.src.n ? a.wavelet[a.m - 1] : (T)0;
    for (int i = tid; i < TZ * TX; i += 256) {
        int lz = i / TX, lx = i - lz * TX;
        int64_t x = x0 + lx, z = z0 + lz;
        if (x >= L.nx || z >= L.nz) continue;
        int64_t q = L.base + z * L.px + x;
        T mu_new = (T)2 * a.mu[q] - a.mum[q] + acc[i];
        a.out[q] = mu_new;
        T Kq = a.K[q];
        if (Kq > (T)0) {
            T d2 = a.pm0[q] - (T)2 * a.pm1[q] + a.pm2[q];
            T srcw = 0;
            for (int s = 0; s < 8 * a.src.n; ++s)
                if (a.src.idx[s] == q) srcw += a.src.w[s];
            d2 -= srcw * wv;
            a.grad[q] += mu_new * ((T)2 * a.dt / sqrt(Kq)) * d2;
            if (a.gw && srcw != (T)0) atomicAdd(&a.gw[a.m - 1], srcw * mu_new);
        }
    }
}

// ---------------------------------------------------------------------------
// setup kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_leap_coef(Layout L, const T* vel, const uint8_t* mask, T dt, T* K) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % L.nx, r = i / L.nx, y = r % L.ny, z = r / L.ny;
        int64_t q = L.idx(x, y, z);
        T c = vel[i];
        K[q] = mask[q] ? dt * dt * c * c : (T)0;
    }
}

template <typename T>
__global__ void k_stag_coef(Layout L, const T* vel, const T* rho, const uint8_t* mp, const uint8_t* mvx,
                            const uint8_t* mvz, T dt, T* kp, T* bx, T* bz) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % L.nx, z = i / L.nx;
        int64_t q = L.idx(x, 0, z);
        T r0 = rho ? rho[i] : (T)1;
        T c = vel[i];
        kp[q] = mp[q] ? dt * r0 * c * c : (T)0;
        T rx = (rho && x + 1 < L.nx) ? rho[i + 1] : r0;
        T rz = (rho && z + 1 < L.nz) ? rho[i + L.nx] : r0;
        bx[q] = mvx[q] ? dt * (T)0.5 * ((T)1 / r0 + (T)1 / rx) : (T)0;
        bz[q] = mvz[q] ? dt * (T)0.5 * ((T)1 / r0 + (T)1 / rz) : (T)0;
    }
}

template <typename T>
__global__ void k_interp_setup(int n, const double* xyz, int ndim, double inv_h, Layout L, const uint8_t* mask,
                               double scale, int64_t* idx, T* w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xi[3] = {0, 0, 0};
        int64_t b[3] = {0, 0, 0};
        double fr[3] = {0, 0, 0};
        int64_t nn[3] = {L.nx, ndim == 3 ? L.ny : L.nz, L.nz};
        for (int a = 0; a < ndim; ++a) {
            xi[a] = xyz[(int64_t)i * ndim + a] * inv_h;
            b[a] = (int64_t)floor(xi[a]);
            fr[a] = xi[a] - (double)b[a];
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
                    q = L.base;
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

template <typename T>
static void stencil_weights(int M, T w2o[5], T c1o[4]) {
    std::vector<double> w2 = ib_central_second(M);
    std::vector<double> c1 = ib_staggered_first(M);
    int H = M / 2;
    for (int k = 0; k < 5; ++k) w2o[k] = k <= H ? (T)w2[H + k] : (T)0;
    for (int k = 0; k < 4; ++k) c1o[k] = k < H ? (T)c1[H + k] : (T)0;   // offset +(k + 1/2)
}

template <typename T>
static OpView<T> view_of(const IbOp& o, const TileBins* b, const Layout& L) {
    OpView<T> v;
    memset(&v, 0, sizeof v);
    if (!b || o.nrows == 0) return v;
    v.row_pad = o.row_pad;
    v.row_ptr = o.row_ptr;
    v.col_pad = o.col_pad;
    v.w = (const T*)(sizeof(T) == 8 ? (const void*)o.w64 : (const void*)o.w32);
    v.tile_ptr = b->tile_ptr;
    v.perm = b->perm;
    v.ntx = (L.nx + b->tx - 1) / b->tx;
    v.nty = (L.ndim == 3 ? (L.ny + b->ty - 1) / b->ty : 1);
    return v;
}

template <typename T>
static OpView<T> view_of_t(const IbOp& o, const TileBins* b, const Layout& L) {
    OpView<T> v;
    memset(&v, 0, sizeof v);
    if (!b || o.t_nrows == 0) return v;
    v.row_pad = o.t_row_pad;
    v.row_ptr = o.t_ptr;
    v.col_pad = o.t_src_off;
    v.w = (const T*)(sizeof(T) == 8 ? (const void*)o.t_w64 : (const void*)o.t_w32);
    v.tile_ptr = b->tile_ptr;
    v.perm = b->perm;
    v.ntx = (L.nx + b->tx - 1) / b->tx;
    v.nty = 1;
    return v;
}

static const int TX2 = 64, TZ2 = 8;

static ib_status check_shot(const ib_table* t, const ib_shot* sh, int precision, double dt, int nt) {
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
        (sh->nrec && (!sh->rec_dev || !sh->traces_dev))) {
        ib_set_error("missing shot arrays");
        return IB_ERR_ARG;
    }
    if (sh->nsrc > 64) {
        ib_set_error("at most 64 sources per shot");
        return IB_ERR_ARG;
    }
    return IB_OK;
}

template <typename T>
struct Geom {
    PointSet<T> src, rec;
};

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
    if (sh->nsrc)
        k_interp_setup<T><<<grid1(sh->nsrc, 64), 64, 0, S.s>>>(sh->nsrc, sh->src_dev, d, 1.0 / t->grid.h, L,
                                                                t->mask_pad[0], scale, si, sw);
    if (sh->nrec)
        k_interp_setup<T><<<grid1(sh->nrec, 64), 64, 0, S.s>>>(sh->nrec, sh->rec_dev, d, 1.0 / t->grid.h, L,
                                                                t->mask_pad[0], 1.0, ri, rw);
    IB_CHECK_LAUNCH("k_interp_setup");
    ib_count_launch("setup");
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

template <typename T>
static ib_status forward_2nd(ib_table* t, const ib_shot* sh, double dt, int nt, void* ckpt, int n_ckpt,
                             cudaStream_t s) {
    const Layout& L = t->L;
    const int d = t->grid.ndim;
    const int M = t->opts.space_order;
    const int H = M / 2;
    Scratch S(s);
    T *p0, *p1, *K;
    TRY(S.alloc(&p0, L.total, true));
    TRY(S.alloc(&p1, L.total, true));
    TRY(S.alloc(&K, L.total, true));
    k_leap_coef<T><<<grid1(L.N, 256), 256, 0, s>>>(L, (const T*)sh->vel_dev, t->mask_pad[0], (T)dt, K);
    IB_CHECK_LAUNCH("k_leap_coef");
    ib_count_launch("setup");
    Geom<T> g;
    TRY(setup_points<T>(t, sh, dt * dt / pow(t->grid.h, d), S, g));
    const TileBins* bins = nullptr;
    int tx = d == 2 ? TX2 : 32, ty = d == 2 ? 1 : 8, tz = d == 2 ? TZ2 : 1;
    if (d == 2) TRY(ib_table_bins(t, 0, false, TX2, 1, TZ2, &bins, s));
    else TRY(ib_table_bins(t, 0, false, 32, 8, 1, &bins, s));
    (void)tx;
    (void)ty;
    (void)tz;
    StepArgs<T> a;
    memset(&a, 0, sizeof a);
    a.L = L;
    {
        T c1u[4];
        stencil_weights<T>(M, a.w2, c1u);
    }
    a.K = K;
    a.inv_h2 = (T)(1.0 / (t->grid.h * t->grid.h));
    a.op = view_of<T>(t->ops[0], bins, L);
    a.src = g.src;
    a.wavelet = (const T*)sh->wavelet_dev;
    a.rec = g.rec;
    a.traces = (T*)sh->traces_dev;
    a.nt = nt;
    const int64_t seg = ckpt ? ckpt_seg(nt, n_ckpt) : 0;
    T* cur = p0;   // p^n
    T* prev = p1;  // p^{n-1}
    dim3 grid2((unsigned)((L.nx + TX2 - 1) / TX2), (unsigned)((L.nz + TZ2 - 1) / TZ2));
    const int zchunk = 32;
    dim3 grid3((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8), (unsigned)((L.nz + zchunk - 1) / zchunk));
    for (int n = 0; n < nt; ++n) {
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
        if (d == 2) {
            PROF_LAUNCH(kname<T>("leap2d_f32", "leap2d_f64"), s, {
                if (H == 1) k_leap2d<T, 1, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
                else if (H == 2) k_leap2d<T, 2, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
                else if (H == 3) k_leap2d<T, 3, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
                else k_leap2d<T, 4, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
            });
        } else {
            dim3 blk(32, 8);
            PROF_LAUNCH(kname<T>("leap3d_f32", "leap3d_f64"), s, {
                if (H == 1) k_leap3d<T, 1><<<grid3, blk, 0, s>>>(a, zchunk);
                else if (H == 2) k_leap3d<T, 2><<<grid3, blk, 0, s>>>(a, zchunk);
                else if (H == 3) k_leap3d<T, 3><<<grid3, blk, 0, s>>>(a, zchunk);
                else k_leap3d<T, 4><<<grid3, blk, 0, s>>>(a, zchunk);
            });
        }
        IB_CHECK_LAUNCH("leapfrog step");
        std::swap(cur, prev);
    }
    if (g.rec.n)
        k_receivers<T><<<grid1(g.rec.n, 256), 256, 0, s>>>(g.rec, cur, (T*)sh->traces_dev, nt, nt - 1);
    IB_CHECK_LAUNCH("k_receivers");
    ib_count_launch("setup");
    return IB_OK;
}

template <typename T>
static ib_status forward_stag(ib_table* t, const ib_shot* sh, double dt, int nt, cudaStream_t s) {
    const Layout& L = t->L;
    const int d = t->grid.ndim;
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
                                                   t->mask_pad[1], t->mask_pad[2], (T)dt, kp, bx, bz);
    IB_CHECK_LAUNCH("k_stag_coef");
    ib_count_launch("setup");
    Geom<T> g;
    TRY(setup_points<T>(t, sh, dt / pow(t->grid.h, d), S, g));
    const TileBins* b[4];
    for (int o = 0; o < 4; ++o) TRY(ib_table_bins(t, o, false, TX2, 1, TZ2, &b[o], s));
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
    a.inv_h = (T)(1.0 / t->grid.h);
    a.gx = view_of<T>(t->ops[0], b[0], L);
    a.gz = view_of<T>(t->ops[1], b[1], L);
    a.dx = view_of<T>(t->ops[2], b[2], L);
    a.dz = view_of<T>(t->ops[3], b[3], L);
    a.src = g.src;
    a.wavelet = (const T*)sh->wavelet_dev;
    a.rec = g.rec;
    a.traces = (T*)sh->traces_dev;
    a.nt = nt;
    dim3 grid2((unsigned)((L.nx + TX2 - 1) / TX2), (unsigned)((L.nz + TZ2 - 1) / TZ2));
    for (int n = 0; n < nt; ++n) {
        a.step = n;
        a.rec_step = n - 1;
        PROF_LAUNCH(kname<T>("stag_v2d_f32", "stag_v2d_f64"), s, {
            if (H == 1) k_stag_v2d<T, 1, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
            else if (H == 2) k_stag_v2d<T, 2, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
            else if (H == 3) k_stag_v2d<T, 3, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
            else k_stag_v2d<T, 4, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
        });
        PROF_LAUNCH(kname<T>("stag_p2d_f32", "stag_p2d_f64"), s, {
            if (H == 1) k_stag_p2d<T, 1, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
            else if (H == 2) k_stag_p2d<T, 2, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
            else if (H == 3) k_stag_p2d<T, 3, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
            else k_stag_p2d<T, 4, TX2, TZ2><<<grid2, 256, 0, s>>>(a);
        });
        IB_CHECK_LAUNCH("staggered step");
    }
    if (g.rec.n) k_receivers<T><<<grid1(g.rec.n, 256), 256, 0, s>>>(g.rec, p, (T*)sh->traces_dev, nt, nt - 1);
    IB_CHECK_LAUNCH("k_receivers");
    ib_count_launch("setup");
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
    return precision == 64 ? forward_stag<double>(t, sh, dt, nt, s) : forward_stag<float>(t, sh, dt, nt, s);
}

// receiver injection table: node -> (receiver, weight), built on the host from the corner lists
template <typename T>
struct InjTable {
    IbOp op;      // row_pad, row_ptr, col_pad = receiver id, w32/w64
    TileBins* bins = nullptr;
};

template <typename T>
static ib_status build_injection(const Layout& L, const PointSet<T>& rec, Scratch& S, OpView<T>& view,
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
    view.col_pad = dcol;
    view.w = dw;
    view.tile_ptr = b.tile_ptr;
    view.perm = b.perm;
    view.ntx = (L.nx + TX2 - 1) / TX2;
    view.nty = 1;
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
    TRY(ib_table_transpose(t, 0, s));
    Scratch S(s);
    T *K, *mu1, *mu2, *grad;
    TRY(S.alloc(&K, L.total, true));
    TRY(S.alloc(&mu1, L.total, true));
    TRY(S.alloc(&mu2, L.total, true));
    TRY(S.alloc(&grad, L.total, true));
    k_leap_coef<T><<<grid1(L.N, 256), 256, 0, s>>>(L, (const T*)sh->vel_dev, t->mask_pad[0], (T)dt, K);
    IB_CHECK_LAUNCH("k_leap_coef");
    ib_count_launch("setup");
    Geom<T> g;
    TRY(setup_points<T>(t, sh, dt * dt / pow(t->grid.h, d), S, g));
    const TileBins* fb = nullptr;
    const TileBins* tb = nullptr;
    TRY(ib_table_bins(t, 0, false, TX2, 1, TZ2, &fb, s));
    TRY(ib_table_bins(t, 0, true, TX2, 1, TZ2, &tb, s));
    std::vector<TileBins> keep;
    OpView<T> inj;
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
    fa.K = K;
    fa.inv_h2 = (T)(1.0 / (t->grid.h * t->grid.h));
    fa.op = view_of<T>(t->ops[0], fb, L);
    fa.src = g.src;
    fa.wavelet = (const T*)sh->wavelet_dev;
    fa.rec.n = 0;
    fa.rec_step = -1;
    fa.nt = nt;
    AdjArgs<T> aa;
    memset(&aa, 0, sizeof aa);
    aa.L = L;
    for (int k = 0; k < 5; ++k) aa.w2[k] = fa.w2[k];
    aa.K = K;
    aa.mask = t->mask_pad[0];
    aa.inv_h2 = fa.inv_h2;
    aa.dt = (T)dt;
    aa.opT = view_of_t<T>(t->ops[0], tb, L);
    aa.inj = inj;
    aa.res = res;
    aa.nt = nt;
    aa.grad = grad;
    aa.src = g.src;
    aa.wavelet = (const T*)sh->wavelet_dev;
    aa.gw = gw;
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
            PROF_LAUNCH(kname<T>("leap2d_f32", "leap2d_f64"), s, {
                if (H == 1) k_leap2d<T, 1, TX2, TZ2><<<grid2, 256, 0, s>>>(fa);
                else if (H == 2) k_leap2d<T, 2, TX2, TZ2><<<grid2, 256, 0, s>>>(fa);
                else if (H == 3) k_leap2d<T, 3, TX2, TZ2><<<grid2, 256, 0, s>>>(fa);
                else k_leap2d<T, 4, TX2, TZ2><<<grid2, 256, 0, s>>>(fa);
            });
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
    IB_CUDA(cudaStreamSynchronize(s));
    for (auto& b : keep) {
        cudaFree(b.tile_ptr);
        cudaFree(b.perm);
    }
    return IB_OK;
}

extern "C" ib_status ib_adjoint(const ib_table* tc, const ib_shot* sh, int32_t precision, double dt, int32_t nt,
                                const void* ckpt, int32_t n_ckpt, const void* residual, void* grad_vel,
                                void* grad_wavelet, void* stream) {
    ib_set_error("");
    TRY(check_shot(tc, sh, precision, dt, nt));
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

extern "C" ib_status ib_forward_batch(const ib_table* const* tables, const ib_shot* shots, int32_t nshot,
                                      int32_t precision, double dt, int32_t nt, void* stream) {
    ib_set_error("");
    if (!tables || !shots || nshot < 1) {
        ib_set_error("empty batch");
        return IB_ERR_ARG;
    }
    for (int i = 0; i < nshot; ++i) TRY(ib_forward(tables[i], &shots[i], precision, dt, nt, nullptr, 0, stream));
    return IB_OK;
}

extern "C" ib_status ib_sync_status(void* stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return ib_cuda_fail(e, "stream", __FILE__, __LINE__);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ib_cuda_fail(e, "device", __FILE__, __LINE__);
    return IB_OK;
}
