// Shared definitions of the immersed-boundary CUDA library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ib.h"

#define IB_MAX_OPS 8

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void ib_set_error(const std::string& msg);
ib_status ib_cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define IB_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ib_cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define IB_CHECK_LAUNCH(what)                                                \
    do {                                                                     \
        cudaError_t e_ = cudaGetLastError();                                 \
        if (e_ != cudaSuccess) return ib_cuda_fail(e_, what, __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// padded wavefield layout
//
// Every field lives in a zero-padded array: H = M/2 zero planes above and
// below, H zero rows before and after each plane (3D), and a row pitch px >=
// nx + H rounded up to 32 elements, so that x - H of one row falls in the
// zero tail of the previous row.  One extra plane (row in 2D) in front keeps
// the most negative stencil offset inside the allocation.  Kernels therefore
// read every stencil neighbour without bounds checks and the zero halo is the
// zero-Dirichlet edge of the model.
// ---------------------------------------------------------------------------
struct Layout {
    int ndim;
    int H;
    int64_t nx, ny, nz;      // logical sizes (ny = 1 in 2D)
    int64_t px;              // row pitch (elements)
    int64_t py;              // rows per plane (3D: ny + 2H; 2D: 1)
    int64_t plane;           // elements per plane (3D: py * px; 2D: px)
    int64_t base;            // padded index of node (0, 0, 0)
    int64_t total;           // elements to allocate
    int64_t N;               // nx * ny * nz

    __host__ __device__ int64_t idx(int64_t x, int64_t y, int64_t z) const {
        return base + z * plane + y * px + x;
    }
    __host__ __device__ int64_t off(int dx, int dy, int dz) const {
        return (int64_t)dz * plane + (int64_t)dy * px + dx;
    }
};

Layout make_layout(int ndim, const int64_t n[3], int H);

// column offset code: dx, dy, dz in [-127, 127] packed in one int32
__host__ __device__ inline int32_t pack_off(int dx, int dy, int dz) {
    return (int32_t)(((uint32_t)(dx & 0xff)) | ((uint32_t)(dy & 0xff) << 8) | ((uint32_t)(dz & 0xff) << 16));
}
__host__ __device__ inline void unpack_off(int32_t c, int& dx, int& dy, int& dz) {
    dx = (int)(int8_t)(c & 0xff);
    dy = (int)(int8_t)((c >> 8) & 0xff);
    dz = (int)(int8_t)((c >> 16) & 0xff);
}

// ---------------------------------------------------------------------------
// correction tables
// ---------------------------------------------------------------------------
struct TileBins {             // rows of one operator binned by step tile
    int tx = 0, ty = 0, tz = 0;
    int64_t ntiles = 0;
    int64_t ntx = 0, nty = 0;
    int32_t* tile_ptr = nullptr;   // [ntiles + 1]
    int32_t* perm = nullptr;       // [nrows] row ids grouped by tile
    // the corrections flattened per tile: entry e of tile t adds
    // w[e] * f[origin(t) + src[e]] to output loc[e] of the tile
    int64_t nent = 0;
    int32_t* ent_ptr = nullptr;    // [ntiles + 1]
    int32_t* ent_loc = nullptr;    // local output index (row-major inside the tile)
    int32_t* ent_src = nullptr;    // source offset from the tile origin (padded index)
    float* ent_w32 = nullptr;
    double* ent_w64 = nullptr;
    // the same entries in compact form (3D step): a 16-bit footprint code
    // (dx + 16) | (dy + 16) << 5 | (dz + 16) << 10 and, for tiles of at most 256
    // nodes, the output slot as one byte: an entry moves 7 bytes (code, slot,
    // FP32 weight) instead of 12
    uint16_t* ent_code = nullptr;  // [nent]
    uint8_t* ent_slot = nullptr;   // [nent]
};

__host__ __device__ inline uint16_t pack_code16(int dx, int dy, int dz) {
    return (uint16_t)((dx + 16) | ((dy + 16) << 5) | ((dz + 16) << 10));
}

// padded index of the first node of a tile (2D: (bx, bz); 3D: (bx, by, z))
__host__ __device__ inline int64_t tile_origin(const Layout& L, const TileBins& b, int64_t tile) {
    int64_t bx = tile % b.ntx;
    int64_t r = tile / b.ntx;
    int64_t by = r % b.nty;
    int64_t bz = r / b.nty;
    if (L.ndim == 2) return L.base + bz * b.tz * L.px + bx * b.tx;
    return L.base + bz * b.tz * L.plane + by * b.ty * L.px + bx * b.tx;
}

void ib_free_bins(TileBins& b);

struct IbOp {
    int64_t nrows = 0, nnz = 0;
    int field_row = 0;            // 0: p nodes, 1 + a: v_a nodes
    int field_col = 0;
    int64_t* row_lin = nullptr;   // unpadded linear node index
    int64_t* row_pad = nullptr;   // padded index
    int64_t* row_ptr = nullptr;   // [nrows + 1]
    int32_t* col_code = nullptr;  // packed (dx, dy, dz)
    int64_t* col_pad = nullptr;   // padded offset (relative to the row node)
    double* w64 = nullptr;
    float* w32 = nullptr;
    int32_t* row_info = nullptr;  // [nrows][4]
    uint16_t* code16 = nullptr;   // [nnz] pack_code16 footprint codes (built on first use)
    std::vector<TileBins> bins;
    // transposed operator (adjoint): rows keyed by column node
    bool have_t = false;
    int64_t t_nrows = 0;
    int64_t* t_row_pad = nullptr;  // column node (padded)
    int64_t* t_ptr = nullptr;
    int64_t* t_src_off = nullptr;  // padded offset from the column node to the row node
    double* t_w64 = nullptr;
    float* t_w32 = nullptr;
    std::vector<TileBins> t_bins;
};

struct ib_table {
    ib_grid grid;
    ib_form form;
    ib_bc bc;
    ib_opts opts;
    Layout L;
    int nops = 0;
    IbOp ops[IB_MAX_OPS];
    uint8_t* mask_pad[4] = {nullptr, nullptr, nullptr, nullptr};   // p, v_0.. interior flags (padded)
    int64_t n_bp = 0, n_fail = 0, n_grown = 0, n_reduced = 0;
    double setup_seconds = 0.0;
    int64_t table_bytes = 0;
    // learned rows (ib_build_stencils_learned)
    double* learned_resid = nullptr;      // [rows of op 0]
    int64_t learned_rows = 0, learned_checked = 0, learned_accepted = 0;
};

// learned-stencil network (ib_mlp.cu)
int ib_mlp_out_count(const ib_mlp* m);
double ib_mlp_out_radius(const ib_mlp* m);
int ib_mlp_ndim(const ib_mlp* m);
int ib_mlp_order(const ib_mlp* m);
const int32_t* ib_mlp_lut(const ib_mlp* m, int* R);
// predictions Y[n][n_out] (FP32) for the given linear node indices
ib_status ib_mlp_predict_nodes(ib_mlp* m, const ib_grid* grid, const double* sdf, const int64_t* nodes,
                               int64_t n, ib_bc bc, float* Y, cudaStream_t s);
// order-preserving compaction: indices i < n with flags[i] != 0 (device list allocated with cudaMalloc)
ib_status ib_compact(const uint8_t* flags, int64_t n, int64_t** out, int64_t* count, cudaStream_t s);

// implemented in ib_build.cu
ib_status ib_table_bins(ib_table* t, int op, bool transposed, int tx, int ty, int tz,
                        const TileBins** out, cudaStream_t s);
ib_status ib_table_transpose(ib_table* t, int op, cudaStream_t s);
ib_status ib_table_code16(ib_table* t, int op, const uint16_t** out, cudaStream_t s);

double ib_wall_seconds();

// launch counting / sampled timing (ib_prof.cu)
struct ProfToken {
    const char* name;
    bool sampled;
    cudaEvent_t e0, e1;
};
void ib_count_launch(const char* name);
ProfToken ib_prof_begin(const char* name, cudaStream_t s);
void ib_prof_end(const ProfToken& t, cudaStream_t s);
