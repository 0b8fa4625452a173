// Stencil constructor: boundary points, IB-row detection, constrained fits in
// FP64 on the GPU, and packing of the correction tables.
//
// Paper sections implemented here:
//   * boundary points = normal projections of grid points onto the surface,
//     kept inside the point-centred unit box; eta cut-off of interior points
//     (boundary-point paragraph of "Approximating Boundary Conditions");
//   * hyperspherical support of radius (order+1)/2 grown until rank(A) equals
//     the number of basis terms, then basis-order reduction (rank and
//     order-reduction paragraphs; 3D first-order example);
//   * A = [Taylor rows of interior points; BC-operator rows at boundary
//     points] (Eq. of the BC dot product), extrapolation B A^+ with zero
//     forcing, folded into the interior stencil ("Reconciliation with the
//     Interior Numerical Discretization");
//   * coupled velocity blocks for the particle-velocity free surface
//     (multi-field section, appendix).
//
// The correction of a modified row is the minimum-norm solution y of
// A^T y = u, u = sum_e w_e a(x_e - x0), restricted to interior rows; this is
// (A^+)^T u.  With R^T R = A^T A (the Cholesky factor of the Gram matrix,
// accumulated over panels of rows so A is never stored) y = A R^{-1} R^{-T} u
// -- the seminormal equations of the minimum-norm problem -- followed by one
// refinement step from the rows of A rebuilt in FP64.  rank(A) = ncol is
// decided from sigma_min / sigma_max of R (A's singular values) estimated by
// inverse and power iteration.  The Householder sweep below serves the
// learned-row check, which needs the row space of the BC rows.
#include <cuda_runtime.h>
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ib_common.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void ib_set_error(const std::string& msg) { g_last_error = msg; }

ib_status ib_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? IB_ERR_OOM : IB_ERR_CUDA;
}

extern "C" const char* ib_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* ib_version(void) { return "ibwave-gb300 0.1"; }

double ib_wall_seconds() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

Layout make_layout(int ndim, const int64_t n[3], int H) {
    Layout L;
    L.ndim = ndim;
    L.H = H;
    L.nx = n[0];
    if (ndim == 2) {
        L.ny = 1;
        L.nz = n[1];
    } else {
        L.ny = n[1];
        L.nz = n[2];
    }
    L.px = ((L.nx + H + 31) / 32) * 32;
    if (ndim == 2) {
        L.py = 1;
        L.plane = L.px;
        L.base = (int64_t)(H + 1) * L.plane;
    } else {
        L.py = L.ny + 2 * H;
        L.plane = L.py * L.px;
        L.base = (int64_t)(H + 1) * L.plane + (int64_t)H * L.px;
    }
    L.total = (L.nz + 2 * H + 1) * L.plane;
    L.N = L.nx * L.ny * L.nz;
    return L;
}

extern "C" void ib_opts_default(ib_opts* o, int32_t M) {
    memset(o, 0, sizeof *o);
    o->space_order = M;
    o->basis_order = 0;
    o->min_order = 2;
    o->radius = 0.0;
    o->growth = 3.0;
    o->eta_p = -1.0;   // by boundary condition: 0.5 free, 0.25 rigid
    o->eta_v = 0.0;
    o->rank_tol = -1.0;   // by boundary condition: 1e-3 free, 1e-2 rigid
}

// ---------------------------------------------------------------------------
// host: 1D stencils from the Taylor system (square solve in long double)
// ---------------------------------------------------------------------------
static std::vector<double> taylor_weights(const std::vector<double>& offs, int deriv) {
    // weights w with sum_j w_j o_j^m / m! = [m == deriv], m = 0..n-1
    int n = (int)offs.size();
    std::vector<long double> A(n * (n + 1));
    for (int m = 0; m < n; ++m) {
        long double fact = 1;
        for (int i = 2; i <= m; ++i) fact *= i;
        for (int j = 0; j < n; ++j) A[m * (n + 1) + j] = powl((long double)offs[j], m) / fact;
        A[m * (n + 1) + n] = (m == deriv) ? 1.0L : 0.0L;
    }
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * (n + 1) + c]) > fabsl(A[p * (n + 1) + c])) p = r;
        for (int j = 0; j <= n; ++j) std::swap(A[c * (n + 1) + j], A[p * (n + 1) + j]);
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            long double f = A[r * (n + 1) + c] / A[c * (n + 1) + c];
            for (int j = 0; j <= n; ++j) A[r * (n + 1) + j] -= f * A[c * (n + 1) + j];
        }
    }
    std::vector<double> w(n);
    for (int j = 0; j < n; ++j) w[j] = (double)(A[j * (n + 1) + n] / A[j * (n + 1) + j]);
    return w;
}

std::vector<double> ib_central_second(int M) {
    std::vector<double> offs;
    for (int k = -M / 2; k <= M / 2; ++k) offs.push_back(k);
    return taylor_weights(offs, 2);
}
std::vector<double> ib_staggered_first(int M) {
    std::vector<double> offs;
    for (int j = 0; j < M; ++j) offs.push_back(j - (M - 1) / 2.0);
    return taylor_weights(offs, 1);
}
static std::vector<double> central_first(int M) {
    std::vector<double> offs;
    for (int k = -M / 2; k <= M / 2; ++k) offs.push_back(k);
    return taylor_weights(offs, 1);
}

// ---------------------------------------------------------------------------
// host: basis multi-indices and boundary-condition templates
// ---------------------------------------------------------------------------
typedef std::array<int, 3> MI;
typedef std::map<MI, double> Op;   // constant-coefficient differential operator

static std::vector<MI> multi_indices(int d, int M) {
    std::vector<MI> out;
    for (int deg = 0; deg <= M; ++deg) {
        std::vector<MI> ks;
        for (int a = 0; a <= deg; ++a)
            for (int b = 0; b <= (d >= 2 ? deg : 0); ++b)
                for (int c = 0; c <= (d >= 3 ? deg : 0); ++c)
                    if (a + b + c == deg) ks.push_back({a, b, c});
        std::sort(ks.begin(), ks.end(), [](const MI& x, const MI& y) { return x > y; });
        out.insert(out.end(), ks.begin(), ks.end());
    }
    return out;
}

static Op op_mul(const Op& p, const Op& q) {
    Op out;
    for (auto& a : p)
        for (auto& b : q) {
            MI k = {a.first[0] + b.first[0], a.first[1] + b.first[1], a.first[2] + b.first[2]};
            out[k] += a.second * b.second;
        }
    return out;
}
static Op op_id() { return Op{{{0, 0, 0}, 1.0}}; }
static Op op_d(int a) {
    MI k = {0, 0, 0};
    k[a] = 1;
    return Op{{k, 1.0}};
}
static Op op_lap(int d) {
    Op o;
    for (int a = 0; a < d; ++a) {
        MI k = {0, 0, 0};
        k[a] = 2;
        o[k] = 1.0;
    }
    return o;
}
static Op op_pow(const Op& p, int k) {
    Op o = op_id();
    for (int i = 0; i < k; ++i) o = op_mul(o, p);
    return o;
}

struct DevTerm {
    int32_t field, axis;
    int32_t alpha[3];
    int32_t pad;
    double coef;
};

struct HostTemplate {           // rows of per-field (axis, operator) terms
    std::vector<std::vector<DevTerm>> rows;
};

static void add_terms(std::vector<DevTerm>& row, const Op& op, int field, int axis) {
    for (auto& t : op) {
        if (t.second == 0.0) continue;
        DevTerm dt;
        dt.field = field;
        dt.axis = axis;
        dt.alpha[0] = t.first[0];
        dt.alpha[1] = t.first[1];
        dt.alpha[2] = t.first[2];
        dt.pad = 0;
        dt.coef = t.second;
        row.push_back(dt);
    }
}

// scalar (pressure) hierarchy: free lap^k p = 0 (2k <= M); rigid n.grad lap^k p = 0 (2k+1 <= M)
// vector (velocity) hierarchy: free lap^k div v = 0 (2k+1 <= M); rigid n.v = 0 and
// n.grad lap^k div v = 0 (2k+2 <= M)
static HostTemplate bc_template(bool vector, ib_bc bc, int d, int M) {
    HostTemplate T;
    Op L = op_lap(d);
    if (!vector) {
        if (bc == IB_FREE) {
            for (int k = 0; 2 * k <= M; ++k) {
                std::vector<DevTerm> row;
                add_terms(row, op_pow(L, k), 0, -1);
                T.rows.push_back(row);
            }
        } else {
            for (int k = 0; 2 * k + 1 <= M; ++k) {
                std::vector<DevTerm> row;
                for (int a = 0; a < d; ++a) add_terms(row, op_mul(op_d(a), op_pow(L, k)), 0, a);
                T.rows.push_back(row);
            }
        }
    } else {
        if (bc == IB_FREE) {
            for (int k = 0; 2 * k + 1 <= M; ++k) {
                std::vector<DevTerm> row;
                for (int a = 0; a < d; ++a) add_terms(row, op_mul(op_d(a), op_pow(L, k)), a, -1);
                T.rows.push_back(row);
            }
        } else {
            std::vector<DevTerm> row0;
            for (int a = 0; a < d; ++a) add_terms(row0, op_id(), a, a);
            T.rows.push_back(row0);
            for (int k = 0; 2 * k + 2 <= M; ++k) {
                std::vector<DevTerm> row;
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b)
                        add_terms(row, op_mul(op_mul(op_d(b), op_d(a)), op_pow(L, k)), a, b);
                T.rows.push_back(row);
            }
            // irrotational acoustic velocity: lap^k (d_i v_j - d_j v_i) = 0, 2k + 1 <= M
            const int pairs2[1][2] = {{0, 1}};
            const int pairs3[3][2] = {{1, 2}, {2, 0}, {0, 1}};
            for (int k = 0; 2 * k + 1 <= M; ++k) {
                int np = d == 2 ? 1 : 3;
                for (int q = 0; q < np; ++q) {
                    int i = d == 2 ? pairs2[q][0] : pairs3[q][0];
                    int j = d == 2 ? pairs2[q][1] : pairs3[q][1];
                    std::vector<DevTerm> row;
                    add_terms(row, op_mul(op_d(i), op_pow(L, k)), j, -1);
                    Op neg = op_mul(op_d(j), op_pow(L, k));
                    for (auto& t : neg) t.second = -t.second;
                    add_terms(row, neg, i, -1);
                    T.rows.push_back(row);
                }
            }
        }
    }
    return T;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#define FIT_MAX_ORDERS 4
#define FIT_MAX_E 32
#define FIT_MAX_SUP 1024
#define FIT_MAX_BP 256
#define FIT_PB 32
#define FIT_THREADS 128
static_assert(FIT_THREADS == 4 * 32 && FIT_PB % 4 == 0, "qr_panel maps 32 columns x 4 row quarters onto the block");
#define FIT_MAX_COL 128

struct OrderDesc {
    int order, T, nbc, pad;
    double r0;
    const int8_t* K;            // [T][3]
    const int32_t* row_start;   // [nbc + 1]
    const DevTerm* terms;
};

struct Geo {
    int ndim;
    int64_t n[3];
    const double* sdf;          // metres, [nz][ny][nx]
    double inv_h;
};

// linear index of a logical node p = (x, [y,] z) (p[2] = 0 in 2D, where p[1] is z)
__device__ __forceinline__ int64_t lin_p(const Geo& g, const int64_t p[3]) {
    return (p[2] * g.n[1] + p[1]) * g.n[0] + p[0];
}
__device__ __forceinline__ bool in_arr(const Geo& g, const int64_t p[3]) {
    for (int a = 0; a < g.ndim; ++a)
        if (p[a] < 0 || p[a] >= g.n[a]) return false;
    return true;
}
__device__ __forceinline__ double sdf_at(const Geo& g, const int64_t p[3]) {
    return g.sdf[lin_p(g, p)];
}
// interior flag of field `kind` (0: p nodes; 1 + a: v_a nodes at j + e_a / 2)
__device__ __forceinline__ bool field_interior(const Geo& g, int kind, const int64_t p[3]) {
    double s = sdf_at(g, p);
    if (kind == 0) return s > 0.0;
    int a = kind - 1;
    int64_t q[3] = {p[0], p[1], p[2]};
    q[a] += 1;
    double s2 = (q[a] < g.n[a]) ? sdf_at(g, q) : s;
    return 0.5 * (s + s2) > 0.0;
}

// ---------------------------------------------------------------------------
// boundary points
// ---------------------------------------------------------------------------
struct BpParams {
    Geo g;
    int M;
    double lim;           // sqrt(d)/2 (grid units)
    const double* cw[5];  // central first-derivative weights of order 2,4,6,8 (index q/2)
};

__constant__ double c_cfirst[5][9];   // [q/2][k + q/2] central first-derivative weights

__device__ bool boundary_point(const Geo& g, int M, int64_t x, int64_t y, int64_t z,
                               double xb[3], double nrm[3]) {
    int64_t p[3];
    p[0] = x;
    if (g.ndim == 3) {
        p[1] = y;
        p[2] = z;
    } else {
        p[1] = z;
        p[2] = 0;
    }
    double s = sdf_at(g, p) * g.inv_h;
    if (fabs(s) > 0.5 * sqrt((double)g.ndim)) return false;
    double gr[3] = {0, 0, 0};
    for (int a = 0; a < g.ndim; ++a) {
        int64_t i = p[a], n = g.n[a];
        int64_t room = i < n - 1 - i ? i : n - 1 - i;
        int64_t q2 = 2 * room < (int64_t)M ? 2 * room : (int64_t)M;
        int q = (int)q2;
        q -= q % 2;
        int64_t qq[3] = {p[0], p[1], p[2]};
        if (q >= 2) {
            double acc = 0.0;
            for (int k = 1; k <= q / 2; ++k) {
                qq[a] = i + k;
                double sp = sdf_at(g, qq);
                qq[a] = i - k;
                double sm = sdf_at(g, qq);
                acc += c_cfirst[q / 2][q / 2 + k] * (sp * g.inv_h - sm * g.inv_h);
            }
            gr[a] = acc;
        } else if (i == 0) {
            qq[a] = 1;
            double s1 = sdf_at(g, qq) * g.inv_h;
            gr[a] = s1 - s;
        } else {
            qq[a] = i - 1;
            double s1 = sdf_at(g, qq) * g.inv_h;
            gr[a] = s - s1;
        }
    }
    double gn = 0.0;
    for (int a = 0; a < g.ndim; ++a) gn += gr[a] * gr[a];
    gn = sqrt(gn);
    if (gn == 0.0) return false;
    double mx = 0.0;
    for (int a = 0; a < 3; ++a) {
        nrm[a] = a < g.ndim ? gr[a] / gn : 0.0;
        double off = -s * nrm[a];
        xb[a] = (double)p[a] + off;
        mx = fmax(mx, fabs(off));
    }
    return mx <= 0.5;
}

__global__ void k_bp_flags(Geo g, int M, uint8_t* flags) {
    int64_t N = g.n[0] * g.n[1] * (g.ndim == 3 ? g.n[2] : 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % g.n[0];
        int64_t r = i / g.n[0];
        int64_t y = g.ndim == 3 ? r % g.n[1] : 0;
        int64_t z = g.ndim == 3 ? r / g.n[1] : r;
        double xb[3], nn[3];
        flags[i] = boundary_point(g, M, x, y, z, xb, nn) ? 1 : 0;
    }
}

__global__ void k_bp_write(Geo g, int M, const int64_t* list, int64_t n, int32_t* bp_index,
                           double* bp_xb, double* bp_n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = list[k];
        int64_t x = i % g.n[0];
        int64_t r = i / g.n[0];
        int64_t y = g.ndim == 3 ? r % g.n[1] : 0;
        int64_t z = g.ndim == 3 ? r / g.n[1] : r;
        double xb[3], nn[3];
        boundary_point(g, M, x, y, z, xb, nn);
        for (int a = 0; a < 3; ++a) {
            bp_xb[3 * k + a] = xb[a];
            bp_n[3 * k + a] = nn[a];
        }
        bp_index[i] = (int32_t)k;
    }
}

// ---------------------------------------------------------------------------
// IB-row detection
// ---------------------------------------------------------------------------
struct RowRule {
    int row_field;           // 0: p node; 1 + a: v_a node
    int nE;
    int Efield[FIT_MAX_E];   // field kind of the stencil point
    int Eoff[FIT_MAX_E][3];  // node offset from the row node
    double Ew[FIT_MAX_E];    // standard weight
};

__global__ void k_row_flags(Geo g, RowRule rule, uint8_t* flags) {
    int64_t N = g.n[0] * g.n[1] * (g.ndim == 3 ? g.n[2] : 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p[3];
        p[0] = i % g.n[0];
        int64_t r = i / g.n[0];
        if (g.ndim == 3) {
            p[1] = r % g.n[1];
            p[2] = r / g.n[1];
        } else {
            p[1] = r;
            p[2] = 0;
        }
        uint8_t f = 0;
        if (field_interior(g, rule.row_field, p)) {
            for (int e = 0; e < rule.nE && !f; ++e) {
                int64_t q[3] = {p[0] + rule.Eoff[e][0], p[1] + rule.Eoff[e][1], p[2] + rule.Eoff[e][2]};
                if (in_arr(g, q) && !field_interior(g, rule.Efield[e], q)) f = 1;
            }
        }
        flags[i] = f;
    }
}

// ---------------------------------------------------------------------------
// the constrained fit (one CTA per IB row)
// ---------------------------------------------------------------------------
struct FitParams {
    Geo g;
    const int32_t* bp_index;
    const double* bp_xb;
    const double* bp_n;
    RowRule rule;
    int nf;
    int fkind[3];             // field kind of each unknown field
    int fshift2[3][3];        // doubled position shift of field nodes
    double feta[3];
    int x0shift2[3];          // doubled expansion-point shift from the row node
    int norders;
    OrderDesc ord[FIT_MAX_ORDERS];
    int ngrow;
    const int8_t* ball_off[3];   // per field: candidate node offsets sorted by distance
    const int32_t* ball_q[3];    // 4 |offset + shift - x0|^2
    int nball[3];
    double rank_tol;
    const int64_t* rows;
    int64_t nrows;
    int ncol_max;
    // outputs
    int32_t* info;              // [nrows][4]
    int32_t* cnt;               // [nrows]
    int64_t* start;             // [nrows]
    int32_t* pool_code;
    int8_t* pool_field;
    double* pool_w;
    unsigned long long* pool_top;
    int64_t pool_cap;
    // learned rows (pred == nullptr: plain fit only)
    const float* pred;          // [nrows][n_out] predicted corrections on the footprint
    int n_out;
    const int32_t* fp_lut;      // footprint index of offset (dx, dy, dz) in [-R, R]^3, or -1
    int fp_R;
    double accept_tol;
    double* resid;              // [nrows] exactness residual of the prediction
    uint8_t* accepted;          // [nrows]
};

__constant__ double c_inv_int[10] = {0.0, 1.0, 0.5, 1.0 / 3.0, 0.25, 0.2, 1.0 / 6.0, 1.0 / 7.0, 0.125, 1.0 / 9.0};

#define PW 9   // powers 0..8 of each coordinate (basis order <= 8)

// pw[a * PW + e] = d_a^e / e!
__device__ __forceinline__ void power_table(const double d[3], double* pw) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = 1.0;
        pw[a * PW] = 1.0;
#pragma unroll
        for (int e = 1; e < PW; ++e) {
            v *= d[a] * c_inv_int[e];
            pw[a * PW + e] = v;
        }
    }
}

// d^alpha of the monomial with exponents k, from a power table
__device__ __forceinline__ double mono_pw(const double* pw, const int8_t* k, const int32_t* alpha) {
    int e0 = k[0] - (alpha ? alpha[0] : 0);
    int e1 = k[1] - (alpha ? alpha[1] : 0);
    int e2 = k[2] - (alpha ? alpha[2] : 0);
    if ((e0 | e1 | e2) < 0) return 0.0;
    return pw[e0] * pw[PW + e1] * pw[2 * PW + e2];
}

struct FitSmem {
    double* R;       // [ncol][ncol]
    double* X;       // [ncol][ncol] = R^{-1} (only when ncol <= 64, else null)
    double* B;       // [PB][ncol]
    double* pwt;     // [PB][3 * PW] power tables of the panel rows
    double* invd;    // [ncol] 1 / R_kk
    double* vec;     // 4 * ncol
    double* bpx;     // [FIT_MAX_BP][3] relative positions
    double* bpn;     // [FIT_MAX_BP][3]
    int32_t* sup;    // packed support: field << 24 | code
    int32_t* bps;    // bp ids
    int* scal;       // misc ints
    double* scald;   // misc doubles
};

__device__ int block_excl_scan(int v, int* tmp, int* total) {
    // tmp: >= 32 ints
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (w == 0) {
        int t = lane < nw ? tmp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) tmp[lane] = t;
    }
    __syncthreads();
    int before = (w > 0 ? tmp[w - 1] : 0) + x - v;
    *total = tmp[nw - 1];
    __syncthreads();
    return before;
}

// position of global row gi of A relative to x0 (grid units)
__device__ __forceinline__ void row_delta(const FitParams& P, const FitSmem& S, int nsup, int nbcrow, int gi,
                                          double d[3]) {
    if (gi < nsup) {
        int32_t c = S.sup[gi];
        int f = c >> 24;
        int dx, dy, dz;
        unpack_off(c & 0xffffff, dx, dy, dz);
        int o[3] = {dx, dy, dz};
        for (int a = 0; a < 3; ++a)
            d[a] = a < P.g.ndim ? 0.5 * (double)(2 * o[a] + P.fshift2[f][a] - P.x0shift2[a]) : 0.0;
    } else {
        int b = (gi - nsup) / nbcrow;
        for (int a = 0; a < 3; ++a) d[a] = S.bpx[3 * b + a];
    }
}

// A entry of global row gi, column col, from the row's power table
__device__ __forceinline__ double a_entry_pw(const FitParams& P, const OrderDesc& od, const FitSmem& S, int nsup,
                                             int nbcrow, int gi, int col, const double* pw) {
    const int f = col / od.T;
    const int k = col - f * od.T;
    const int8_t* K = od.K + 3 * k;
    if (gi < nsup) return ((S.sup[gi] >> 24) == f) ? mono_pw(pw, K, nullptr) : 0.0;
    const int j = gi - nsup;
    const int b = j / nbcrow;
    const int r = j - b * nbcrow;
    const double* nn = S.bpn + 3 * b;
    double v = 0.0;
    for (int t = od.row_start[r]; t < od.row_start[r + 1]; ++t) {
        const DevTerm& tm = od.terms[t];
        if (tm.field != f) continue;
        const double c = tm.coef * (tm.axis >= 0 ? nn[tm.axis] : 1.0);
        if (c != 0.0) v += c * mono_pw(pw, K, tm.alpha);
    }
    return v;
}

// rows row0 .. row0 + PB - 1 of A into the panel B (zero rows past m)
__device__ void build_panel(const FitParams& P, const OrderDesc& od, const FitSmem& S, int nsup,
                            int nbcrow, int m, int row0, int ncol) {
    for (int i = threadIdx.x; i < FIT_PB; i += blockDim.x) {
        int gi = row0 + i;
        double d[3] = {0.0, 0.0, 0.0};
        if (gi < m) row_delta(P, S, nsup, nbcrow, gi, d);
        power_table(d, S.pwt + i * 3 * PW);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < FIT_PB * ncol; idx += blockDim.x) {
        int i = idx / ncol, col = idx - i * ncol;
        int gi = row0 + i;
        S.B[idx] = gi < m ? a_entry_pw(P, od, S, nsup, nbcrow, gi, col, S.pwt + i * 3 * PW) : 0.0;
    }
}

// Householder sweep: [R; B] -> [R'; 0]
__device__ void qr_panel(const FitSmem& S, int ncol) {
    double* R = S.R;
    double* B = S.B;
    for (int k = 0; k < ncol; ++k) {
        if (threadIdx.x < 32) {
            int lane = threadIdx.x;
            double b = lane < FIT_PB ? B[lane * ncol + k] : 0.0;
            double ss = b * b;
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            if (lane == 0) {
                double rkk = R[k * ncol + k];
                if (ss == 0.0) {
                    S.scald[0] = 0.0;   // tau
                } else {
                    double nrm = sqrt(rkk * rkk + ss);
                    double alpha = rkk >= 0.0 ? -nrm : nrm;
                    double v0 = rkk - alpha;
                    S.scald[0] = 2.0 / (v0 * v0 + ss);
                    S.scald[1] = v0;
                    S.scald[2] = alpha;
                }
            }
        }
        __syncthreads();
        double tau = S.scald[0];
        if (tau != 0.0) {
            // thread = (column c of 32, row quarter g of the panel): four lanes share a
            // column, so every lane of a warp carries a column while columns remain
            const double v0 = S.scald[1];
            const int g = threadIdx.x & 3, c = threadIdx.x >> 2;
            const int wfirst = (threadIdx.x >> 5) * 8;       // first column offset of this warp
            double bk[FIT_PB / 4];
#pragma unroll
            for (int r = 0; r < FIT_PB / 4; ++r) bk[r] = B[(g * (FIT_PB / 4) + r) * ncol + k];
            for (int jb = k + 1; jb + wfirst < ncol; jb += 32) {
                const int j = jb + c;
                const bool act = j < ncol;
                double w = 0.0;
                if (act) {
#pragma unroll
                    for (int r = 0; r < FIT_PB / 4; ++r) w += bk[r] * B[(g * (FIT_PB / 4) + r) * ncol + j];
                    if (g == 0) w += v0 * R[k * ncol + j];
                }
                w += __shfl_xor_sync(0xffffffffu, w, 1);
                w += __shfl_xor_sync(0xffffffffu, w, 2);
                if (act) {
                    w *= tau;
                    if (g == 0) R[k * ncol + j] -= v0 * w;
#pragma unroll
                    for (int r = 0; r < FIT_PB / 4; ++r) B[(g * (FIT_PB / 4) + r) * ncol + j] -= bk[r] * w;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && tau != 0.0) R[k * ncol + k] = S.scald[2];
        __syncthreads();
    }
}

// Gram matrix of the fit, streamed over panels: G += B^T B (upper triangle of G,
// kept in S.R).  Every (i, j) pair is owned by one thread, so a panel needs no
// block-wide step per column.
__device__ void gram_panel(const FitSmem& S, int ncol) {
    const int np = ncol * (ncol + 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        int i = 0, rem = p;                         // p -> (i, j), i <= j, row by row
        while (rem >= ncol - i) {
            rem -= ncol - i;
            ++i;
        }
        const int j = i + rem;
        double a = 0.0;
#pragma unroll 8
        for (int r = 0; r < FIT_PB; ++r) a += S.B[r * ncol + i] * S.B[r * ncol + j];
        S.R[i * ncol + j] += a;
    }
}

// Upper Cholesky factor R of G in place (R^T R = G = A^T A, so R has A's
// singular values).  A non-positive pivot (columns dependent at working
// precision) leaves a zero diagonal and a zero row, which the rank test reads
// as singular.
__device__ void chol_upper(const FitSmem& S, int n) {
    double* R = S.R;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double piv = R[k * n + k];
            S.scald[0] = piv > 0.0 ? sqrt(piv) : 0.0;
        }
        __syncthreads();
        const double rkk = S.scald[0];
        const double inv = rkk > 0.0 ? 1.0 / rkk : 0.0;
        for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) R[k * n + j] *= inv;
        if (threadIdx.x == 0) R[k * n + k] = rkk;
        __syncthreads();
        const int w = n - k - 1;
        for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
            const int i = k + 1 + q / w, j = k + 1 + q % w;
            if (j >= i) R[i * n + j] -= R[k * n + i] * R[k * n + j];
        }
        __syncthreads();
    }
}

// warp-level triangular solves on R (row-major, upper), vector in shared memory
__device__ void warp_solve_RT(const double* R, const double* invd, int n, double* x) {   // R^T w = x
    int lane = threadIdx.x & 31;
    for (int k = 0; k < n; ++k) {
        double wk = x[k] * invd[k];
        __syncwarp();
        if (lane == 0) x[k] = wk;
        for (int i = k + 1 + lane; i < n; i += 32) x[i] -= R[k * n + i] * wk;
        __syncwarp();
    }
}
__device__ void warp_solve_R(const double* R, const double* invd, int n, double* x) {    // R y = x
    int lane = threadIdx.x & 31;
    for (int k = n - 1; k >= 0; --k) {
        double yk = x[k] * invd[k];
        __syncwarp();
        if (lane == 0) x[k] = yk;
        for (int i = lane; i < k; i += 32) x[i] -= R[i * n + k] * yk;
        __syncwarp();
    }
}

// rank decisions whose first estimate lies in (tol, RANK_RECHECK tol] are
// estimated again with RANK_ITERS_FINE iterations
#define RANK_RECHECK 2.0
#define RANK_ITERS_FINE 600

// sigma_min / sigma_max of R by power and inverse iteration in one warp, in
// FP32 (the rank decision needs a few digits; GB300's FP64 pipe is the
// constructor's bottleneck).  x, y: scratch of n floats each.
__device__ float warp_norm_f(const float* x, int n) {
    float s = 0.f;
    for (int i = threadIdx.x & 31; i < n; i += 32) s += x[i] * x[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return sqrtf(s);
}
__device__ double warp_cond_ratio(const double* R, const double* invd, int n, double* xd, double* yd,
                                  int it_max, int it_min) {
    const int lane = threadIdx.x & 31;
    float* x = (float*)xd;
    float* y = (float*)yd;
    for (int i = lane; i < n; i += 32) x[i] = rsqrtf((float)n);
    __syncwarp();
    float smax2 = 0.f;
    for (int it = 0; it < it_max; ++it) {
        for (int i = lane; i < n; i += 32) {
            float s = 0.f;
            for (int j = i; j < n; ++j) s += (float)R[i * n + j] * x[j];
            y[i] = s;
        }
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            float s = 0.f;
            for (int i = 0; i <= j; ++i) s += (float)R[i * n + j] * y[i];
            x[j] = s;
        }
        __syncwarp();
        const float nr = warp_norm_f(x, n);
        if (!(nr > 0.f) || !(nr < 3e38f)) return 0.0;
        smax2 = nr;
        for (int i = lane; i < n; i += 32) x[i] /= nr;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) x[i] = rsqrtf((float)n) * (1.f + 0.01f * (float)(i % 7));
    __syncwarp();
    const float nx0 = warp_norm_f(x, n);
    for (int i = lane; i < n; i += 32) x[i] /= nx0;
    __syncwarp();
    float smin2 = 0.f;
    for (int it = 0; it < it_min; ++it) {
        // R^T w = x, then R x' = w (forward and back substitution, one warp)
        for (int k = 0; k < n; ++k) {
            const float wk = x[k] * (float)invd[k];
            __syncwarp();
            if (lane == 0) x[k] = wk;
            for (int i = k + 1 + lane; i < n; i += 32) x[i] -= (float)R[k * n + i] * wk;
            __syncwarp();
        }
        for (int k = n - 1; k >= 0; --k) {
            const float yk = x[k] * (float)invd[k];
            __syncwarp();
            if (lane == 0) x[k] = yk;
            for (int i = lane; i < k; i += 32) x[i] -= (float)R[i * n + k] * yk;
            __syncwarp();
        }
        const float nr = warp_norm_f(x, n);
        if (!(nr < 3e38f) || nr == 0.f) return 0.0;
        smin2 = 1.f / nr;
        for (int i = lane; i < n; i += 32) x[i] /= nr;
        __syncwarp();
    }
    return sqrt((double)smin2 / (double)smax2);
}

// The same estimate from an FP32 copy of R packed by rows (upper triangle):
// element (i, j), j >= i, at rs(i) + j - i with rs(i) = i (2n - i + 1) / 2.
__device__ __forceinline__ int packed_rs(int i, int n) { return i * (2 * n - i + 1) / 2; }
__device__ double warp_cond_ratio_packed(const float* Rp, const float* invf, int n, double* xd, double* yd,
                                         int it_max, int it_min) {
    const int lane = threadIdx.x & 31;
    float* x = (float*)xd;
    float* y = (float*)yd;
    for (int i = lane; i < n; i += 32) x[i] = rsqrtf((float)n);
    __syncwarp();
    float smax2 = 0.f;
    for (int it = 0; it < it_max; ++it) {
        for (int i = lane; i < n; i += 32) {
            const float* row = Rp + packed_rs(i, n) - i;
            float s = 0.f;
            for (int j = i; j < n; ++j) s += row[j] * x[j];
            y[i] = s;
        }
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            float s = 0.f;
            int rs = 0;
            for (int i = 0; i <= j; ++i) {
                s += Rp[rs + j - i] * y[i];
                rs += n - i;
            }
            x[j] = s;
        }
        __syncwarp();
        const float nr = warp_norm_f(x, n);
        if (!(nr > 0.f) || !(nr < 3e38f)) return 0.0;
        smax2 = nr;
        for (int i = lane; i < n; i += 32) x[i] /= nr;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) x[i] = rsqrtf((float)n) * (1.f + 0.01f * (float)(i % 7));
    __syncwarp();
    const float nx0 = warp_norm_f(x, n);
    for (int i = lane; i < n; i += 32) x[i] /= nx0;
    __syncwarp();
    float smin2 = 0.f;
    for (int it = 0; it < it_min; ++it) {
        for (int k = 0; k < n; ++k) {
            const float wk = x[k] * invf[k];
            __syncwarp();
            if (lane == 0) x[k] = wk;
            const float* row = Rp + packed_rs(k, n) - k;
            for (int i = k + 1 + lane; i < n; i += 32) x[i] -= row[i] * wk;
            __syncwarp();
        }
        for (int k = n - 1; k >= 0; --k) {
            const float yk = x[k] * invf[k];
            __syncwarp();
            if (lane == 0) x[k] = yk;
            for (int i = lane; i < k; i += 32) x[i] -= Rp[packed_rs(i, n) + k - i] * yk;
            __syncwarp();
        }
        const float nr = warp_norm_f(x, n);
        if (!(nr < 3e38f) || nr == 0.f) return 0.0;
        smin2 = 1.f / nr;
        for (int i = lane; i < n; i += 32) x[i] /= nr;
        __syncwarp();
    }
    return sqrt((double)smin2 / (double)smax2);
}

// X = R^{-1} (upper triangular): thread j back-substitutes column j
__device__ void tri_inverse(const double* R, const double* invd, double* X, int n) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        for (int i = n - 1; i > j; --i) X[i * n + j] = 0.0;
        X[j * n + j] = invd[j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= j; ++k) s += R[i * n + k] * X[k * n + j];
            X[i * n + j] = -s * invd[i];
        }
    }
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

__device__ float block_sum_f(float v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = (double)v;
    __syncthreads();
    float t = 0.f;
    for (int i = 0; i < nw; ++i) t += (float)red[i];
    return t;
}

// largest singular value of an upper-triangular M (row-major, FP64 in shared
// memory) by power iteration on M^T M in FP32: the rank decision needs a few
// digits, and GB300's FP64 pipe is the constructor's bottleneck
__device__ float block_sigma_max(const float* M, int n, float* v, float* w, double* red, int iters) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = 1.f + 0.01f * (float)(i % 5);
    __syncthreads();
    float t0 = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t0 += v[i] * v[i];
    float nrm = sqrtf(block_sum_f(t0, red));
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] /= nrm;
    __syncthreads();
    float lam = 0.f;
    for (int it = 0; it < iters; ++it) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            float t = 0.f;
            for (int j = i; j < n; ++j) t += M[i * n + j] * v[j];
            w[i] = t;
        }
        __syncthreads();
        float t2 = 0.f;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            float t = 0.f;
            for (int i = 0; i <= j; ++i) t += M[i * n + j] * w[i];
            v[j] = t;
            t2 += t * t;
        }
        lam = sqrtf(block_sum_f(t2, red));
        if (!(lam > 0.f) || !(lam < 3e38f)) return lam;
        for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] /= lam;
        __syncthreads();
    }
    return sqrtf(lam);
}

// z = X (X^T y) with X = R^{-1}: the solve (R^T R) z = y by two triangular matvecs
__device__ void x_solve(const double* X, int n, const double* y, double* t, double* z) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i <= j; ++i) s += X[i * n + j] * y[i];
        t[j] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int j = i; j < n; ++j) s += X[i * n + j] * t[j];
        z[i] = s;
    }
    __syncthreads();
}

// right-hand side u = sum_e w_e a(x_e - x0) over the exterior stencil points
__device__ void fit_rhs(const FitParams& P, const OrderDesc& od, unsigned emask, int ncol, double* u) {
    for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
        int f = col / od.T;
        int k = col - f * od.T;
        double acc = 0.0;
        for (int e = 0; e < P.rule.nE; ++e) {
            if (!((emask >> e) & 1u)) continue;
            int ef = P.rule.Efield[e];
            int fi = 0;   // unknown field index of this stencil point's field kind
            for (int ff = 0; ff < P.nf; ++ff)
                if (P.fkind[ff] == ef) fi = ff;
            if (fi != f) continue;
            double d[3], pw[3 * PW];
            for (int a = 0; a < 3; ++a)
                d[a] = a < P.g.ndim ? 0.5 * (double)(2 * P.rule.Eoff[e][a] + P.fshift2[f][a] - P.x0shift2[a]) : 0.0;
            power_table(d, pw);
            acc += P.rule.Ew[e] * mono_pw(pw, od.K + 3 * k, nullptr);
        }
        u[col] = acc;
    }
}

// reserve n pool entries (whole block); false on overflow
__device__ bool pool_alloc(const FitParams& P, const FitSmem& S, int n, int64_t* start) {
    if (threadIdx.x == 0) {
        unsigned long long st = atomicAdd(P.pool_top, (unsigned long long)n);
        S.scal[1] = (int)(st & 0x7fffffff);
        S.scal[2] = (int)(st >> 31);
    }
    __syncthreads();
    *start = ((int64_t)S.scal[2] << 31) | (int64_t)S.scal[1];
    __syncthreads();
    return *start + n <= P.pool_cap;
}

__device__ __forceinline__ int fp_index(const FitParams& P, int32_t code) {
    int dx, dy, dz;
    unpack_off(code & 0xffffff, dx, dy, dz);
    const int R = P.fp_R, W = 2 * R + 1;
    if (dx < -R || dx > R || dy < -R || dy > R || dz < -R || dz > R) return -1;
    return P.fp_lut[((dz + R) * W + (dy + R)) * W + (dx + R)];
}

// Exactness residual of the predicted correction of this row at the current
// support: v = A_I^T c - u, projected on the null space of the BC rows (the
// orthogonal complement of the row space of R_B, A_B = Q_B R_B), relative to
// |u|.  The row space is spanned by classical Gram-Schmidt with one
// re-orthogonalisation over the rows of R_B, dropping rows whose remainder is
// below 1e-10 of the largest row norm.  +inf when the prediction does not
// apply (a support node off the footprint, coupled fields, too many columns)
// or cannot be checked (the BC rows have full column rank, so no basis
// polynomial satisfies them and exactness says nothing).
__device__ double learned_residual(const FitParams& P, const OrderDesc& od, const FitSmem& S, int64_t row,
                                   int nsup, int nbcrow, int m, int ncol, unsigned emask) {
    const int ncm = P.ncol_max;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x == 0) S.scal[4] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nsup; i += blockDim.x)
        if (fp_index(P, S.sup[i]) < 0) S.scal[4] = 1;
    __syncthreads();
    if (S.scal[4] != 0 || S.X == nullptr || P.nf != 1) return INFINITY;
    double* u = S.vec;
    double* v = S.vec + ncm;
    double* w = S.vec + 2 * ncm;
    double* dots = S.vec + 3 * ncm;
    double* rn = S.invd;                  // row norms^2 of R_B
    double* red = S.scald + 4;
    fit_rhs(P, od, emask, ncol, u);
    __syncthreads();
    for (int col = threadIdx.x; col < ncol; col += blockDim.x) v[col] = -u[col];
    // v += A_I^T c
    double* ci = S.scald + 16;            // [FIT_PB]
    for (int row0 = 0; row0 < nsup; row0 += FIT_PB) {
        build_panel(P, od, S, nsup, nbcrow, nsup, row0, ncol);
        for (int i = threadIdx.x; i < FIT_PB; i += blockDim.x)
            ci[i] = row0 + i < nsup ? (double)P.pred[row * P.n_out + fp_index(P, S.sup[row0 + i])] : 0.0;
        __syncthreads();
        for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
            double a = 0.0;
            for (int i = 0; i < FIT_PB; ++i) a += S.B[i * ncol + col] * ci[i];
            v[col] += a;
        }
        __syncthreads();
    }
    // R_B: streamed QR of the boundary-condition rows only
    for (int i = threadIdx.x; i < ncol * ncol; i += blockDim.x) S.R[i] = 0.0;
    __syncthreads();
    for (int row0 = nsup; row0 < m; row0 += FIT_PB) {
        build_panel(P, od, S, nsup, nbcrow, m, row0, ncol);
        __syncthreads();
        qr_panel(S, ncol);
    }
    for (int i = warp; i < ncol; i += nwarp) {
        double a = 0.0;
        for (int j = lane; j < ncol; j += 32) a += S.R[i * ncol + j] * S.R[i * ncol + j];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) rn[i] = a;
    }
    __syncthreads();
    double rmax2 = 0.0;
    for (int i = 0; i < ncol; ++i) rmax2 = fmax(rmax2, rn[i]);
    const double thr2 = 1e-20 * rmax2;
    double* X = S.X;                      // orthonormal rows
    int nq = 0;
    for (int i = 0; i < ncol; ++i) {
        if (!(rn[i] > thr2)) continue;
        for (int j = threadIdx.x; j < ncol; j += blockDim.x) w[j] = S.R[i * ncol + j];
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = warp; q < nq; q += nwarp) {
                double a = 0.0;
                for (int j = lane; j < ncol; j += 32) a += X[q * ncol + j] * w[j];
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) dots[q] = a;
            }
            __syncthreads();
            for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
                double a = w[j];
                for (int q = 0; q < nq; ++q) a -= dots[q] * X[q * ncol + j];
                w[j] = a;
            }
            __syncthreads();
        }
        double part = 0.0;
        for (int j = threadIdx.x; j < ncol; j += blockDim.x) part += w[j] * w[j];
        const double n2 = block_sum(part, red);
        if (n2 > thr2) {
            const double inv = 1.0 / sqrt(n2);
            for (int j = threadIdx.x; j < ncol; j += blockDim.x) X[nq * ncol + j] = w[j] * inv;
            ++nq;
        }
        __syncthreads();
    }
    // no polynomial of the basis satisfies every boundary condition: the test
    // has no content, so the prediction cannot be verified
    if (nq >= ncol) return INFINITY;
    // remove the row-space part of v (twice)
    for (int pass = 0; pass < 2; ++pass) {
        for (int q = warp; q < nq; q += nwarp) {
            double a = 0.0;
            for (int j = lane; j < ncol; j += 32) a += X[q * ncol + j] * v[j];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) dots[q] = a;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
            double a = v[j];
            for (int q = 0; q < nq; ++q) a -= dots[q] * X[q * ncol + j];
            v[j] = a;
        }
        __syncthreads();
    }
    double pv = 0.0, pu = 0.0;
    for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
        pv += v[j] * v[j];
        pu += u[j] * u[j];
    }
    const double nv2 = block_sum(pv, red);
    const double nu2 = block_sum(pu, red);
    return sqrt(nv2) / (nu2 > 0.0 ? sqrt(nu2) : 1.0);
}

__global__ void __launch_bounds__(FIT_THREADS) k_fit(FitParams P) {
    extern __shared__ double smem_d[];
    const int ncm = P.ncol_max;
    FitSmem S;
    S.R = smem_d;
    S.X = ncm <= 64 ? S.R + ncm * ncm : nullptr;
    S.B = S.R + ncm * ncm * (ncm <= 64 ? 2 : 1);
    S.pwt = S.B + FIT_PB * ncm;
    S.invd = S.pwt + FIT_PB * 3 * PW;
    S.vec = S.invd + ncm;
    S.bpx = S.vec + 4 * ncm;
    S.bpn = S.bpx + 3 * FIT_MAX_BP;
    S.scald = S.bpn + 3 * FIT_MAX_BP;     // [48]: 0..7 scalars, 4..7 block_sum scratch, 16..47 panel dots
    S.sup = (int32_t*)(S.scald + 48);
    S.bps = S.sup + FIT_MAX_SUP;
    S.scal = S.bps + FIT_MAX_BP;          // [0..63]
    int* scan_tmp = S.scal + 16;

    for (int64_t row = blockIdx.x; row < P.nrows; row += gridDim.x) {
        const int64_t lin = P.rows[row];
        int64_t node[3];
        node[0] = lin % P.g.n[0];
        int64_t rr = lin / P.g.n[0];
        if (P.g.ndim == 3) {
            node[1] = rr % P.g.n[1];
            node[2] = rr / P.g.n[1];
        } else {
            node[1] = rr;
            node[2] = 0;
        }
        // expansion point (grid units)
        double x0[3];
        for (int a = 0; a < 3; ++a) x0[a] = (double)node[a] + 0.5 * P.x0shift2[a];

        // exterior stencil points -> mask of E entries (same for every order/radius)
        if (threadIdx.x == 0) {
            unsigned em = 0;
            for (int e = 0; e < P.rule.nE; ++e) {
                int64_t q[3] = {node[0] + P.rule.Eoff[e][0], node[1] + P.rule.Eoff[e][1],
                                node[2] + P.rule.Eoff[e][2]};
                if (in_arr(P.g, q) && !field_interior(P.g, P.rule.Efield[e], q)) em |= 1u << e;
            }
            S.scal[0] = (int)em;
        }
        __syncthreads();
        const unsigned emask = (unsigned)S.scal[0];

        int status = 1, used_order = 0, used_r2 = 0, used_nbp = 0, nsup_final = 0;
        bool done = false;
        for (int oi = 0; oi < P.norders && !done; ++oi) {
            const OrderDesc& od = P.ord[oi];
            const int ncol = P.nf * od.T;
            for (int gstep = 0; gstep <= P.ngrow && !done; ++gstep) {
                const double r = od.r0 + 0.5 * gstep;
                const int qlim = (int)floor(4.0 * r * r + 1e-9);
                // ---- interior support (deterministic order: field, then distance)
                int nsup = 0;
                bool overflow = false;
                for (int f = 0; f < P.nf; ++f) {
                    const int8_t* bo = P.ball_off[f];
                    const int32_t* bq = P.ball_q[f];
                    for (int c0 = 0; c0 < P.nball[f]; c0 += blockDim.x) {
                        if (bq[c0] > qlim) break;   // sorted by distance: the rest is outside r
                        int c = c0 + threadIdx.x;
                        int ok = 0;
                        int32_t code = 0;
                        if (c < P.nball[f] && bq[c] <= qlim) {
                            int o[3] = {bo[3 * c], bo[3 * c + 1], bo[3 * c + 2]};
                            int64_t q[3] = {node[0] + o[0], node[1] + o[1], node[2] + o[2]};
                            if (in_arr(P.g, q) && field_interior(P.g, P.fkind[f], q)) {
                                ok = 1;
                                // eta exclusion: a boundary point strictly inside the 2 eta box
                                double eta = P.feta[f];
                                if (eta > 0.0) {
                                    double pos[3];
                                    for (int a = 0; a < 3; ++a) pos[a] = (double)q[a] + 0.5 * P.fshift2[f][a];
                                    int lo[3], hi[3];
                                    for (int a = 0; a < 3; ++a) {
                                        if (a < P.g.ndim) {
                                            lo[a] = (int)ceil(pos[a] - 0.5 - eta - 1e-12);
                                            hi[a] = (int)floor(pos[a] + 0.5 + eta + 1e-12);
                                        } else {
                                            lo[a] = hi[a] = 0;
                                        }
                                    }
                                    for (int zz = lo[2]; zz <= hi[2] && ok; ++zz)
                                        for (int yy = lo[1]; yy <= hi[1] && ok; ++yy)
                                            for (int xx = lo[0]; xx <= hi[0] && ok; ++xx) {
                                                int64_t w[3] = {xx, yy, zz};
                                                if (!in_arr(P.g, w)) continue;
                                                int32_t b = P.bp_index[lin_p(P.g, w)];
                                                if (b < 0) continue;
                                                double mx = 0.0;
                                                for (int a = 0; a < P.g.ndim; ++a)
                                                    mx = fmax(mx, fabs(P.bp_xb[3 * b + a] - pos[a]));
                                                if (mx < eta) ok = 0;
                                            }
                                }
                            }
                            code = (f << 24) | pack_off(o[0], o[1], o[2]);
                        }
                        int tot;
                        int pos = block_excl_scan(ok, scan_tmp, &tot);
                        if (ok && nsup + pos < FIT_MAX_SUP) S.sup[nsup + pos] = code;
                        nsup += tot;
                    }
                }
                if (nsup > FIT_MAX_SUP) overflow = true;
                // ---- boundary points within r of x0 (owner order)
                int nbp = 0;
                {
                    int lo[3], hi[3];
                    int64_t span = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (a < P.g.ndim) {
                            lo[a] = (int)ceil(x0[a] - r - 0.5 - 1e-12);
                            hi[a] = (int)floor(x0[a] + r + 0.5 + 1e-12);
                        } else {
                            lo[a] = hi[a] = 0;
                        }
                        span *= (hi[a] - lo[a] + 1);
                    }
                    int wx = hi[0] - lo[0] + 1, wy = hi[1] - lo[1] + 1;
                    for (int64_t c0 = 0; c0 < span; c0 += blockDim.x) {
                        int64_t c = c0 + threadIdx.x;
                        int ok = 0;
                        int32_t b = -1;
                        if (c < span) {
                            int xx = lo[0] + (int)(c % wx);
                            int yy = lo[1] + (int)((c / wx) % wy);
                            int zz = lo[2] + (int)(c / ((int64_t)wx * wy));
                            int64_t w[3] = {xx, yy, zz};
                            if (in_arr(P.g, w)) {
                                b = P.bp_index[lin_p(P.g, w)];
                                if (b >= 0) {
                                    double d2 = 0.0;
                                    for (int a = 0; a < P.g.ndim; ++a) {
                                        double dd = P.bp_xb[3 * b + a] - x0[a];
                                        d2 += dd * dd;
                                    }
                                    ok = d2 <= r * r + 1e-9;
                                }
                            }
                        }
                        int tot;
                        int pos = block_excl_scan(ok, scan_tmp, &tot);
                        if (ok && nbp + pos < FIT_MAX_BP) S.bps[nbp + pos] = b;
                        nbp += tot;
                    }
                }
                if (nbp > FIT_MAX_BP) overflow = true;
                if (overflow) {
                    status = 4;
                    done = true;
                    break;
                }
                for (int i = threadIdx.x; i < nbp; i += blockDim.x) {
                    int b = S.bps[i];
                    for (int a = 0; a < 3; ++a) {
                        S.bpx[3 * i + a] = a < P.g.ndim ? P.bp_xb[3 * b + a] - x0[a] : 0.0;
                        S.bpn[3 * i + a] = P.bp_n[3 * b + a];
                    }
                }
                const int nbcrow = od.nbc;
                const int m = nsup + nbp * nbcrow;
                if (P.pred && oi == 0 && gstep == 0) {
                    // ---- learned row: keep the prediction if it is exact on the BC-satisfying basis
                    const double rho = learned_residual(P, od, S, row, nsup, nbcrow, m, ncol, emask);
                    if (threadIdx.x == 0) P.resid[row] = rho;
                    if (rho <= P.accept_tol && rho < INFINITY) {
                        int64_t start;
                        if (!pool_alloc(P, S, nsup, &start)) {
                            status = 3;
                            done = true;
                            break;
                        }
                        for (int i = threadIdx.x; i < nsup; i += blockDim.x) {
                            P.pool_code[start + i] = S.sup[i] & 0xffffff;
                            P.pool_field[start + i] = (int8_t)(S.sup[i] >> 24);
                            P.pool_w[start + i] = (double)P.pred[row * P.n_out + fp_index(P, S.sup[i])];
                        }
                        if (threadIdx.x == 0) {
                            P.start[row] = start;
                            P.accepted[row] = 1;
                        }
                        status = 0;
                        used_order = od.order;
                        used_r2 = (int)lrint(2.0 * r);
                        used_nbp = nbp;
                        nsup_final = nsup;
                        done = true;
                        break;
                    }
                    __syncthreads();
                }
                if (m < ncol) continue;
                // ---- R with R^T R = A^T A: Gram matrix streamed over panels (A is never
                // stored), then its Cholesky factor.  The seminormal solve below and its
                // FP64 refinement from the rebuilt rows of A recover the accuracy.
                for (int i = threadIdx.x; i < ncol * ncol; i += blockDim.x) S.R[i] = 0.0;
                __syncthreads();
                for (int row0 = 0; row0 < m; row0 += FIT_PB) {
                    build_panel(P, od, S, nsup, nbcrow, m, row0, ncol);
                    __syncthreads();
                    gram_panel(S, ncol);
                    __syncthreads();
                }
                chol_upper(S, ncol);
                // ---- rank test: sigma_min / sigma_max of R
                for (int k = threadIdx.x; k < ncol; k += blockDim.x) {
                    double rkk = S.R[k * ncol + k];
                    S.invd[k] = rkk != 0.0 ? 1.0 / rkk : 0.0;
                }
                if (threadIdx.x == 0) S.scal[3] = 0;
                __syncthreads();
                for (int k = threadIdx.x; k < ncol; k += blockDim.x)
                    if (S.invd[k] == 0.0) S.scal[3] = 1;
                __syncthreads();
                double ratio = 0.0;
                const bool singular = S.scal[3] != 0;
                if (!singular) {
                    if (S.X) {
                        tri_inverse(S.R, S.invd, S.X, ncol);
                        __syncthreads();
                        float* fv = (float*)S.vec;          // 2 * ncm floats in vec[0 .. ncm)
                        // FP32 copies in the (now free) panel buffer: ncol^2 floats fit in
                        // FIT_PB * ncm doubles for ncm <= 64, and one conversion per
                        // element keeps the FP64 pipe out of the iterations
                        float* fm = (float*)S.B;
                        for (int i = threadIdx.x; i < ncol * ncol; i += blockDim.x) fm[i] = (float)S.R[i];
                        __syncthreads();
                        // Power iteration approaches each sigma_max from below, so the
                        // estimated ratio is never below the true one: a fit it rejects is
                        // rank deficient, and an acceptance close to the threshold is
                        // checked again with RANK_ITERS_FINE iterations.
                        for (int pass = 0; pass < 2; ++pass) {
                            const int iters = pass ? RANK_ITERS_FINE : 30;
                            if (pass) {
                                for (int i = threadIdx.x; i < ncol * ncol; i += blockDim.x) fm[i] = (float)S.R[i];
                                __syncthreads();
                            }
                            float smax = block_sigma_max(fm, ncol, fv, fv + ncm, S.scald + 4, iters);
                            __syncthreads();
                            for (int i = threadIdx.x; i < ncol * ncol; i += blockDim.x) fm[i] = (float)S.X[i];
                            __syncthreads();
                            float sinv = block_sigma_max(fm, ncol, fv, fv + ncm, S.scald + 4, iters);
                            __syncthreads();
                            ratio = (smax > 0.f && sinv > 0.f && sinv < 3e38f) ? 1.0 / ((double)smax * (double)sinv)
                                                                               : 0.0;
                            if (!(ratio > P.rank_tol && ratio < RANK_RECHECK * P.rank_tol)) break;
                        }
                    } else {
                        // packed FP32 copy of R (and 1/R_kk) in the free panel buffer when it fits
                        const int npk = ncol * (ncol + 1) / 2;
                        const bool packed = (npk + ncol) * 4 <= FIT_PB * ncm * 8;
                        float* rp = (float*)S.B;
                        if (packed) {
                            for (int i = threadIdx.x; i < ncol; i += blockDim.x) {
                                const int rs = packed_rs(i, ncol) - i;
                                for (int j = i; j < ncol; ++j) rp[rs + j] = (float)S.R[i * ncol + j];
                                rp[npk + i] = (float)S.invd[i];
                            }
                            __syncthreads();
                        }
                        if (threadIdx.x < 32) {
                            // the same one-sided estimate; near the threshold, again with more iterations
                            double rr = 0.0;
                            for (int pass = 0; pass < 2; ++pass) {
                                const int im = pass ? RANK_ITERS_FINE : 24, in = pass ? RANK_ITERS_FINE : 40;
                                rr = packed ? warp_cond_ratio_packed(rp, rp + npk, ncol, S.vec, S.vec + ncm, im, in)
                                            : warp_cond_ratio(S.R, S.invd, ncol, S.vec, S.vec + ncm, im, in);
                                if (!(rr > P.rank_tol && rr < RANK_RECHECK * P.rank_tol)) break;
                            }
                            if (threadIdx.x == 0) S.scald[4] = rr;
                        }
                        __syncthreads();
                        ratio = S.scald[4];
                    }
                }
                __syncthreads();
                if (!(ratio > P.rank_tol)) continue;
                // ---- right-hand side u = sum_e w_e a(x_e - x0)
                double* u = S.vec;              // [ncol]
                double* z = S.vec + ncm;        // [ncol]
                double* rho = S.vec + 2 * ncm;  // [ncol]
                double* tv = S.vec + 3 * ncm;   // [ncol] scratch
                fit_rhs(P, od, emask, ncol, u);
                __syncthreads();
                for (int col = threadIdx.x; col < ncol; col += blockDim.x) z[col] = u[col];
                __syncthreads();
                if (S.X) {
                    x_solve(S.X, ncol, u, tv, z);
                } else {
                    if (threadIdx.x < 32) {
                        warp_solve_RT(S.R, S.invd, ncol, z);
                        warp_solve_R(S.R, S.invd, ncol, z);
                    }
                    __syncthreads();
                }
                // ---- one refinement step: rho = u - A^T (A z); z += (R^T R)^{-1} rho
                for (int col = threadIdx.x; col < ncol; col += blockDim.x) rho[col] = u[col];
                __syncthreads();
                double* s_i = S.scald + 16;      // [FIT_PB]
                for (int row0 = 0; row0 < m; row0 += FIT_PB) {
                    build_panel(P, od, S, nsup, nbcrow, m, row0, ncol);
                    __syncthreads();
                    for (int i = threadIdx.x >> 5; i < FIT_PB; i += blockDim.x >> 5) {
                        double sacc = 0.0;
                        for (int col = threadIdx.x & 31; col < ncol; col += 32) sacc += S.B[i * ncol + col] * z[col];
                        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                        if ((threadIdx.x & 31) == 0) s_i[i] = sacc;
                    }
                    __syncthreads();
                    for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
                        double acc = 0.0;
                        for (int i = 0; i < FIT_PB; ++i) acc += S.B[i * ncol + col] * s_i[i];
                        rho[col] -= acc;
                    }
                    __syncthreads();
                }
                if (S.X) {
                    x_solve(S.X, ncol, rho, tv, u);          // u <- correction (u no longer needed)
                    for (int col = threadIdx.x; col < ncol; col += blockDim.x) z[col] += u[col];
                } else {
                    if (threadIdx.x < 32) {
                        warp_solve_RT(S.R, S.invd, ncol, rho);
                        warp_solve_R(S.R, S.invd, ncol, rho);
                    }
                    __syncthreads();
                    for (int col = threadIdx.x; col < ncol; col += blockDim.x) z[col] += rho[col];
                }
                __syncthreads();
                // ---- output: y_i = A_i z for interior rows
                int64_t start;
                if (!pool_alloc(P, S, nsup, &start)) {
                    status = 3;   // pool overflow: re-run with a larger pool
                    done = true;
                    break;
                }
                for (int row0 = 0; row0 < nsup; row0 += FIT_PB) {
                    build_panel(P, od, S, nsup, nbcrow, nsup, row0, ncol);
                    __syncthreads();
                    for (int i = threadIdx.x >> 5; i < FIT_PB && row0 + i < nsup; i += blockDim.x >> 5) {
                        double sacc = 0.0;
                        for (int col = threadIdx.x & 31; col < ncol; col += 32) sacc += S.B[i * ncol + col] * z[col];
                        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                        if ((threadIdx.x & 31) == 0) {
                            const int gi = row0 + i;
                            P.pool_code[start + gi] = S.sup[gi] & 0xffffff;
                            P.pool_field[start + gi] = (int8_t)(S.sup[gi] >> 24);
                            P.pool_w[start + gi] = sacc;
                        }
                    }
                    __syncthreads();
                }
                if (threadIdx.x == 0) P.start[row] = start;
                status = 0;
                used_order = od.order;
                used_r2 = (int)lrint(2.0 * r);
                used_nbp = nbp;
                nsup_final = nsup;
                done = true;
            }
        }
        if (threadIdx.x == 0) {
            P.info[4 * row + 0] = used_r2;
            P.info[4 * row + 1] = used_order;
            P.info[4 * row + 2] = used_nbp;
            P.info[4 * row + 3] = status;
            P.cnt[row] = status == 0 ? nsup_final : 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// packing
// ---------------------------------------------------------------------------
__global__ void k_pack(int64_t nrows, const int32_t* cnt, const int64_t* start, const int64_t* out_ptr_all,
                       const int32_t* pool_code, const int8_t* pool_field, const double* pool_w,
                       int field, int nf, int32_t* out_code, double* out_w64, float* out_w32,
                       int64_t* out_pad, Layout L, int64_t* out_cnt_field) {
    // out_ptr_all: per-row start within this field's CSR (exclusive scan of per-field counts)
    for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
        int n = cnt[row];
        int64_t s = start[row];
        int64_t o = out_ptr_all[row];
        // entries of this field keep their order within the row
        __shared__ int base;
        if (threadIdx.x == 0) base = 0;
        __syncthreads();
        for (int i0 = 0; i0 < n; i0 += blockDim.x) {
            int i = i0 + threadIdx.x;
            int mine = (i < n && pool_field[s + i] == field) ? 1 : 0;
            unsigned bal = __ballot_sync(0xffffffffu, mine);
            // blockDim == 32 for this kernel
            int pos = __popc(bal & ((1u << (threadIdx.x & 31)) - 1));
            if (mine) {
                int64_t dst = o + base + pos;
                int32_t c = pool_code[s + i];
                out_code[dst] = c;
                double w = pool_w[s + i];
                out_w64[dst] = w;
                out_w32[dst] = (float)w;
                int dx, dy, dz;
                unpack_off(c, dx, dy, dz);
                out_pad[dst] = L.off(dx, dy, dz);
            }
            __syncwarp();
            if (threadIdx.x == 0) base += __popc(bal);
            __syncwarp();
        }
        __syncthreads();
    }
}

__global__ void k_count_field(int64_t nrows, const int32_t* cnt, const int64_t* start,
                              const int8_t* pool_field, int field, int64_t* out) {
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < nrows;
         row += (int64_t)gridDim.x * blockDim.x) {
        int n = cnt[row];
        int64_t s = start[row];
        int64_t c = 0;
        for (int i = 0; i < n; ++i) c += pool_field[s + i] == field;
        out[row] = c;
    }
}

__global__ void k_row_pad(int64_t n, const int64_t* lin, Layout L, int64_t* pad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = lin[i];
        int64_t x = l % L.nx;
        int64_t r = l / L.nx;
        int64_t y = r % L.ny;
        int64_t z = r / L.ny;
        pad[i] = L.idx(x, y, z);
    }
}

__global__ void k_masks(Geo g, Layout L, int nfield, uint8_t* m0, uint8_t* m1, uint8_t* m2, uint8_t* m3) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p[3];
        int64_t x = i % L.nx;
        int64_t r = i / L.nx;
        int64_t y = r % L.ny;
        int64_t z = r / L.ny;
        p[0] = x;
        if (g.ndim == 3) {
            p[1] = y;
            p[2] = z;
        } else {
            p[1] = z;
            p[2] = 0;
        }
        int64_t q = L.idx(x, y, z);
        uint8_t* ms[4] = {m0, m1, m2, m3};
        for (int f = 0; f < nfield; ++f) ms[f][q] = field_interior(g, f, p) ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
template <class T>
static ib_status dalloc(T** p, int64_t n) {
    *p = nullptr;
    if (n <= 0) n = 1;
    IB_CUDA(cudaMalloc((void**)p, sizeof(T) * (size_t)n));
    return IB_OK;
}
#define TRY(x)                          \
    do {                                \
        ib_status st_ = (x);            \
        if (st_ != IB_OK) return st_;   \
    } while (0)

static ib_status compact(const uint8_t* flags, int64_t n, int64_t** out, int64_t* count, cudaStream_t s) {
    int64_t* d_out = nullptr;
    int64_t* d_cnt = nullptr;
    TRY(dalloc(&d_out, n));
    TRY(dalloc(&d_cnt, 1));
    thrust::counting_iterator<int64_t> it(0);
    size_t tmp = 0;
    IB_CUDA(cub::DeviceSelect::Flagged(nullptr, tmp, it, flags, d_out, d_cnt, n, s));
    void* d_tmp = nullptr;
    IB_CUDA(cudaMalloc(&d_tmp, tmp + 16));
    IB_CUDA(cub::DeviceSelect::Flagged(d_tmp, tmp, it, flags, d_out, d_cnt, n, s));
    IB_CUDA(cudaMemcpyAsync(count, d_cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    IB_CUDA(cudaStreamSynchronize(s));
    cudaFree(d_tmp);
    cudaFree(d_cnt);
    *out = d_out;
    return IB_OK;
}

ib_status ib_compact(const uint8_t* flags, int64_t n, int64_t** out, int64_t* count, cudaStream_t s) {
    return compact(flags, n, out, count, s);
}

static ib_status excl_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    size_t tmp = 0;
    IB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, in, out, n, s));
    void* d_tmp = nullptr;
    IB_CUDA(cudaMalloc(&d_tmp, tmp + 16));
    IB_CUDA(cub::DeviceScan::ExclusiveSum(d_tmp, tmp, in, out, n, s));
    IB_CUDA(cudaStreamSynchronize(s));
    cudaFree(d_tmp);
    return IB_OK;
}

static int grid_for(int64_t n, int bs) {
    int64_t g = (n + bs - 1) / bs;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    ib_status alloc(T** p, int64_t n) {
        TRY(dalloc(p, n));
        ptrs.push_back((void*)*p);
        return IB_OK;
    }
};

// Sorted candidate offsets of one field: |o + frac| <= rmax (frac doubled in frac2)
static void make_ball(int d, const int frac2[3], double rmax, std::vector<int8_t>& off, std::vector<int32_t>& q) {
    int R = (int)ceil(rmax) + 1;
    int qmax = (int)floor(4.0 * rmax * rmax + 1e-9);
    struct E {
        int q, z, y, x;
    };
    std::vector<E> v;
    for (int z = (d >= 3 ? -R : 0); z <= (d >= 3 ? R : 0); ++z)
        for (int y = (d >= 2 ? -R : 0); y <= (d >= 2 ? R : 0); ++y)
            for (int x = -R; x <= R; ++x) {
                int o[3] = {x, y, z};
                int qq = 0;
                for (int a = 0; a < d; ++a) {
                    int t = 2 * o[a] + frac2[a];
                    qq += t * t;
                }
                if (qq <= qmax) v.push_back({qq, z, y, x});
            }
    std::sort(v.begin(), v.end(), [](const E& a, const E& b) {
        if (a.q != b.q) return a.q < b.q;
        if (a.z != b.z) return a.z < b.z;
        if (a.y != b.y) return a.y < b.y;
        return a.x < b.x;
    });
    off.clear();
    q.clear();
    for (auto& e : v) {
        // logical order (x, y, z) with the 2D second axis in slot 1
        off.push_back((int8_t)e.x);
        off.push_back((int8_t)e.y);
        off.push_back((int8_t)e.z);
        q.push_back(e.q);
    }
}

struct FitKind {
    RowRule rule;
    int nf;
    int fkind[3];
    int fshift2[3][3];
    double feta[3];
    int x0shift2[3];
    bool vector_bc;
    // learned rows (second-order form): network, the geometry it reads, acceptance threshold
    ib_mlp* mlp = nullptr;
    const ib_grid* grid = nullptr;
    const double* sdf = nullptr;
    double accept_tol = -1.0;
};

// Build the fits of one kind and return the packed per-field CSR tables.
// the fit results of the rows (pool entries per row, info) packed into the
// table's CSR operators, one per field
static ib_status pack_pool(ib_table* t, const FitKind& fk, const int64_t* rows, int64_t nrows, const int32_t* info,
                           const int32_t* cnt, const int64_t* start, const int32_t* pool_code,
                           const int8_t* pool_field, const double* pool_w, int op_first, cudaStream_t s,
                           DevBuf& tmp) {
    const Layout& L = t->L;
    for (int f = 0; f < fk.nf; ++f) {
        IbOp& op = t->ops[op_first + f];
        op.nrows = nrows;
        op.field_row = fk.rule.row_field;
        op.field_col = fk.fkind[f];
        int64_t *fc, *fptr;
        TRY(tmp.alloc(&fc, nrows + 1));
        TRY(dalloc(&op.row_ptr, nrows + 1));
        IB_CUDA(cudaMemsetAsync(fc, 0, sizeof(int64_t) * (nrows + 1), s));
        if (nrows) {
            k_count_field<<<grid_for(nrows, 256), 256, 0, s>>>(nrows, cnt, start, pool_field, f, fc);
            IB_CHECK_LAUNCH("k_count_field");
            ib_count_launch("setup");
        }
        TRY(excl_scan(fc, op.row_ptr, nrows + 1, s));
        fptr = op.row_ptr;
        int64_t nnz = 0;
        IB_CUDA(cudaMemcpy(&nnz, op.row_ptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost));
        op.nnz = nnz;
        TRY(dalloc(&op.col_code, nnz));
        TRY(dalloc(&op.col_pad, nnz));
        TRY(dalloc(&op.w64, nnz));
        TRY(dalloc(&op.w32, nnz));
        TRY(dalloc(&op.row_lin, nrows));
        TRY(dalloc(&op.row_pad, nrows));
        TRY(dalloc(&op.row_info, 4 * nrows));
        if (nrows) {
            k_pack<<<grid_for(nrows, 32), 32, 0, s>>>(nrows, cnt, start, fptr, pool_code, pool_field, pool_w, f,
                                                       fk.nf, op.col_code, op.w64, op.w32, op.col_pad, L, nullptr);
            IB_CHECK_LAUNCH("k_pack");
            ib_count_launch("setup");
            IB_CUDA(cudaMemcpyAsync(op.row_lin, rows, sizeof(int64_t) * nrows, cudaMemcpyDeviceToDevice, s));
            IB_CUDA(cudaMemcpyAsync(op.row_info, info, 16 * nrows, cudaMemcpyDeviceToDevice, s));
            k_row_pad<<<grid_for(nrows, 256), 256, 0, s>>>(nrows, rows, L, op.row_pad);
            IB_CHECK_LAUNCH("k_row_pad");
            ib_count_launch("setup");
        }
        IB_CUDA(cudaStreamSynchronize(s));
        t->table_bytes += nnz * (4 + 8 + 8 + 4) + nrows * (8 + 8 + 8 + 16);
    }
    return IB_OK;
}

static ib_status run_fit(ib_table* t, const Geo& g, const FitKind& fk, const int32_t* bp_index,
                         const double* bp_xb, const double* bp_n, int op_first, cudaStream_t s,
                         DevBuf& tmp) {
    const int d = g.ndim;
    const Layout& L = t->L;
    // rows
    uint8_t* flags = nullptr;
    TRY(tmp.alloc(&flags, L.N));
    k_row_flags<<<grid_for(L.N, 256), 256, 0, s>>>(g, fk.rule, flags);
    IB_CHECK_LAUNCH("k_row_flags");
            ib_count_launch("setup");
    int64_t* rows = nullptr;
    int64_t nrows = 0;
    TRY(compact(flags, L.N, &rows, &nrows, s));
    tmp.ptrs.push_back(rows);
    // per-order tables
    int basis = t->opts.basis_order;
    std::vector<int> orders;
    for (int o = basis; o >= t->opts.min_order && (int)orders.size() < FIT_MAX_ORDERS; o -= 2) orders.push_back(o);
    FitParams P;
    memset(&P, 0, sizeof P);
    P.g = g;
    P.bp_index = bp_index;
    P.bp_xb = bp_xb;
    P.bp_n = bp_n;
    P.rule = fk.rule;
    P.nf = fk.nf;
    for (int f = 0; f < 3; ++f) {
        P.fkind[f] = fk.fkind[f];
        P.feta[f] = fk.feta[f];
        for (int a = 0; a < 3; ++a) P.fshift2[f][a] = fk.fshift2[f][a];
        P.x0shift2[f] = fk.x0shift2[f];
    }
    P.norders = (int)orders.size();
    P.ngrow = (int)lrint(t->opts.growth / 0.5);
    P.rank_tol = t->opts.rank_tol;
    double rmax = 0.0;
    int ncol_max = 0;
    for (int oi = 0; oi < P.norders; ++oi) {
        int Mp = orders[oi];
        std::vector<MI> K = multi_indices(d, Mp);
        HostTemplate ht = bc_template(fk.vector_bc, t->bc, d, Mp);
        std::vector<int8_t> kk;
        for (auto& m : K) {
            kk.push_back((int8_t)m[0]);
            kk.push_back((int8_t)m[1]);
            kk.push_back((int8_t)m[2]);
        }
        std::vector<int32_t> rs(1, 0);
        std::vector<DevTerm> terms;
        for (auto& row : ht.rows) {
            terms.insert(terms.end(), row.begin(), row.end());
            rs.push_back((int32_t)terms.size());
        }
        int8_t* dK;
        int32_t* drs;
        DevTerm* dterms;
        TRY(tmp.alloc(&dK, (int64_t)kk.size()));
        TRY(tmp.alloc(&drs, (int64_t)rs.size()));
        TRY(tmp.alloc(&dterms, (int64_t)terms.size()));
        IB_CUDA(cudaMemcpy(dK, kk.data(), kk.size(), cudaMemcpyHostToDevice));
        IB_CUDA(cudaMemcpy(drs, rs.data(), rs.size() * 4, cudaMemcpyHostToDevice));
        IB_CUDA(cudaMemcpy(dterms, terms.data(), terms.size() * sizeof(DevTerm), cudaMemcpyHostToDevice));
        OrderDesc& od = P.ord[oi];
        od.order = Mp;
        od.T = (int)K.size();
        od.nbc = (int)ht.rows.size();
        od.r0 = (t->opts.radius > 0.0 && oi == 0) ? t->opts.radius : (Mp + 1) / 2.0;
        od.K = dK;
        od.row_start = drs;
        od.terms = dterms;
        rmax = std::max(rmax, od.r0 + 0.5 * P.ngrow);
        ncol_max = std::max(ncol_max, fk.nf * od.T);
    }
    if (ncol_max > FIT_MAX_COL) {
        ib_set_error("basis too large for the GPU constructor (columns > 128)");
        return IB_ERR_ARG;
    }
    P.ncol_max = std::max(ncol_max, FIT_PB);
    for (int f = 0; f < fk.nf; ++f) {
        int frac2[3];
        for (int a = 0; a < 3; ++a) frac2[a] = fk.fshift2[f][a] - fk.x0shift2[a];
        std::vector<int8_t> off;
        std::vector<int32_t> q;
        make_ball(d, frac2, rmax, off, q);
        int8_t* doff;
        int32_t* dq;
        TRY(tmp.alloc(&doff, (int64_t)off.size()));
        TRY(tmp.alloc(&dq, (int64_t)q.size()));
        IB_CUDA(cudaMemcpy(doff, off.data(), off.size(), cudaMemcpyHostToDevice));
        IB_CUDA(cudaMemcpy(dq, q.data(), q.size() * 4, cudaMemcpyHostToDevice));
        P.ball_off[f] = doff;
        P.ball_q[f] = dq;
        P.nball[f] = (int)q.size();
    }
    // learned predictions of every row (checked inside k_fit)
    uint8_t* accepted = nullptr;
    if (fk.mlp) {
        if (fk.nf != 1 || P.ncol_max > 64 || fabs(P.ord[0].r0 - ib_mlp_out_radius(fk.mlp)) > 1e-12) {
            ib_set_error("learned stencils: the network's output radius must equal the first support radius "
                         "of a single-field fit with at most 64 columns");
            return IB_ERR_ARG;
        }
        TRY(dalloc(&t->learned_resid, std::max<int64_t>(nrows, 1)));
        t->learned_rows = nrows;
        IB_CUDA(cudaMemsetAsync(t->learned_resid, 0xff, sizeof(double) * std::max<int64_t>(nrows, 1), s));
        TRY(tmp.alloc(&accepted, std::max<int64_t>(nrows, 1)));
        float* pred = nullptr;
        const int n_out = ib_mlp_out_count(fk.mlp);
        TRY(tmp.alloc(&pred, std::max<int64_t>(nrows, 1) * n_out));
        if (nrows) TRY(ib_mlp_predict_nodes(fk.mlp, fk.grid, fk.sdf, rows, nrows, t->bc, pred, s));
        P.pred = pred;
        P.n_out = n_out;
        P.fp_lut = ib_mlp_lut(fk.mlp, &P.fp_R);
        P.accept_tol = fk.accept_tol;
        P.resid = t->learned_resid;
        P.accepted = accepted;
    }
    // outputs
    int32_t *info, *cnt;
    int64_t* start;
    TRY(tmp.alloc(&info, 4 * std::max<int64_t>(nrows, 1)));
    TRY(tmp.alloc(&cnt, std::max<int64_t>(nrows, 1)));
    TRY(tmp.alloc(&start, std::max<int64_t>(nrows, 1)));
    IB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * std::max<int64_t>(nrows, 1), s));
    int64_t cap = std::max<int64_t>(nrows * 48 * fk.nf, 1024);
    int32_t* pool_code;
    int8_t* pool_field;
    double* pool_w;
    unsigned long long* top;
    TRY(tmp.alloc(&top, 1));
    std::vector<int64_t> redo;
    for (int attempt = 0; attempt < 3; ++attempt) {
        TRY(tmp.alloc(&pool_code, cap));
        TRY(tmp.alloc(&pool_field, cap));
        TRY(tmp.alloc(&pool_w, cap));
        IB_CUDA(cudaMemsetAsync(top, 0, sizeof(unsigned long long), s));
        if (accepted) IB_CUDA(cudaMemsetAsync(accepted, 0, std::max<int64_t>(nrows, 1), s));
        P.rows = rows;
        P.nrows = nrows;
        P.info = info;
        P.cnt = cnt;
        P.start = start;
        P.pool_code = pool_code;
        P.pool_field = pool_field;
        P.pool_w = pool_w;
        P.pool_top = top;
        P.pool_cap = cap;
        size_t ncm = (size_t)P.ncol_max;
        size_t shm = sizeof(double) * (ncm * ncm * (ncm <= 64 ? 2 : 1) + (size_t)FIT_PB * ncm + FIT_PB * 3 * PW +
                                       ncm + 4 * ncm + 6 * FIT_MAX_BP + 48) +
                     sizeof(int32_t) * (FIT_MAX_SUP + FIT_MAX_BP + 64);
        IB_CUDA(cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        if (nrows > 0) {
            int blocks = (int)std::min<int64_t>(nrows, 152 * 16);
            k_fit<<<blocks, FIT_THREADS, shm, s>>>(P);
            IB_CHECK_LAUNCH("k_fit");
            ib_count_launch("setup");
        }
        IB_CUDA(cudaStreamSynchronize(s));
        // pool overflow?
        std::vector<int32_t> hinfo(4 * nrows);
        if (nrows) IB_CUDA(cudaMemcpy(hinfo.data(), info, 16 * nrows, cudaMemcpyDeviceToHost));
        int64_t over = 0;
        for (int64_t i = 0; i < nrows; ++i) over += hinfo[4 * i + 3] == 3;
        if (!over) break;
        cap *= 4;   // rerun everything with a larger pool (rare)
    }
    // statistics
    std::vector<int32_t> hinfo(4 * nrows);
    if (nrows) IB_CUDA(cudaMemcpy(hinfo.data(), info, 16 * nrows, cudaMemcpyDeviceToHost));
    int64_t nfail = 0;
    for (int64_t i = 0; i < nrows; ++i) {
        int st = hinfo[4 * i + 3];
        if (st != 0) ++nfail;
        else {
            if (hinfo[4 * i + 1] != orders[0]) t->n_reduced++;
            else if (hinfo[4 * i + 0] != (int)lrint(2.0 * P.ord[0].r0)) t->n_grown++;
        }
    }
    t->n_fail += nfail;
    if (accepted && nrows) {
        std::vector<uint8_t> hacc(nrows);
        std::vector<double> hres(nrows);
        IB_CUDA(cudaMemcpy(hacc.data(), accepted, nrows, cudaMemcpyDeviceToHost));
        IB_CUDA(cudaMemcpy(hres.data(), t->learned_resid, 8 * nrows, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nrows; ++i) {
            t->learned_accepted += hacc[i] != 0;
            t->learned_checked += std::isfinite(hres[i]) ? 1 : 0;
        }
    }
    // pack per field
    return pack_pool(t, fk, rows, nrows, info, cnt, start, pool_code, pool_field, pool_w, op_first, s, tmp);
}

// ---------------------------------------------------------------------------
// Per-axis 1D extrapolation ("Reduction to 1D": the paper's method with a 1D
// basis on each grid line, the sub-case it relates to Mulder's scheme), free
// surface.  One thread per IB row.  For each axis and each side of the row's
// axial stencil that reaches in-array exterior nodes: the boundary is where the
// SDF, interpolated linearly between the last interior node and the first
// exterior node on that side, crosses zero; the interior points are the P/2
// nodes on the line closest to it at more than eta; the 1D Taylor basis of order
// P = M (lowered by 2 while the line holds too few such nodes) is fitted to them
// and to p = 0, p'' = 0, .., p^(P) = 0 at the boundary (a square system, solved
// by Gaussian elimination with partial pivoting in FP64); every exterior node of
// that side takes the extrapolated value.  Entries go to row-owned pool slots.
// ---------------------------------------------------------------------------
#define FIT1D_MAXE 32

struct Fit1dParams {
    Geo g;
    int M;
    double eta;
    double w2[9];           // central second-derivative weights, offsets -H .. H
    const int64_t* rows;
    int64_t nrows;
    int32_t* info;          // [nrows][4]
    int32_t* cnt;
    int64_t* start;
    int32_t* pool_code;
    int8_t* pool_field;
    double* pool_w;
};

// inverse of the (n x n) row-major matrix A (n <= 9) into Ai; false if singular
__device__ bool small_inverse(double* A, double* Ai, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ai[i * 9 + j] = i == j ? 1.0 : 0.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * 9 + c]) > fabs(A[piv * 9 + c])) piv = r;
        if (A[piv * 9 + c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                double t = A[c * 9 + j];
                A[c * 9 + j] = A[piv * 9 + j];
                A[piv * 9 + j] = t;
                t = Ai[c * 9 + j];
                Ai[c * 9 + j] = Ai[piv * 9 + j];
                Ai[piv * 9 + j] = t;
            }
        const double inv = 1.0 / A[c * 9 + c];
        for (int j = 0; j < n; ++j) {
            A[c * 9 + j] *= inv;
            Ai[c * 9 + j] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r * 9 + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[r * 9 + j] -= f * A[c * 9 + j];
                Ai[r * 9 + j] -= f * Ai[c * 9 + j];
            }
        }
    }
    return true;
}

__global__ void __launch_bounds__(128) k_fit1d(Fit1dParams P) {
    const Geo& g = P.g;
    const int H = P.M / 2;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < P.nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lin = P.rows[r];
        int64_t p[3] = {lin % g.n[0], 0, 0};
        if (g.ndim == 2) {
            p[1] = lin / g.n[0];
        } else {
            p[1] = (lin / g.n[0]) % g.n[1];
            p[2] = lin / (g.n[0] * g.n[1]);
        }
        int32_t code[FIT1D_MAXE];
        double wsum[FIT1D_MAXE];
        int ne = 0;
        int pmin = P.M;
        bool bad = false;
        for (int a = 0; a < g.ndim; ++a)
            for (int sg = 1; sg >= -1; sg -= 2) {
                unsigned ext = 0;
                for (int k = 1; k <= H; ++k) {
                    int64_t q[3] = {p[0], p[1], p[2]};
                    q[a] += sg * k;
                    if (in_arr(g, q) && !(sdf_at(g, q) > 0.0)) ext |= 1u << k;
                }
                if (!ext) continue;
                const int kb = __ffs(ext) - 1;
                int64_t qi[3] = {p[0], p[1], p[2]}, qe[3] = {p[0], p[1], p[2]};
                qi[a] += sg * (kb - 1);
                qe[a] += sg * kb;
                const double s1 = sdf_at(g, qi), s2 = sdf_at(g, qe);
                const double ub = (kb - 1) + s1 / (s1 - s2);
                int cand[4];
                int nc = 0;
                for (int u = kb - 1; nc < H; --u) {
                    int64_t q[3] = {p[0], p[1], p[2]};
                    q[a] += sg * u;
                    if (!in_arr(g, q) || !(sdf_at(g, q) > 0.0)) break;
                    if (ub - u > P.eta) cand[nc++] = u;
                }
                int Pd = P.M;
                while (Pd > 0 && nc < Pd / 2) Pd -= 2;
                const int need = Pd / 2, n = Pd + 1;
                pmin = min(pmin, Pd);
                if (need == 0) continue;   // order 0: the extrapolant is zero
                // rows: basis u^m / m! at the interior points, then the even derivatives at ub
                double A[81], Ai[81], fact[9];
                fact[0] = 1.0;
                for (int m = 1; m < n; ++m) fact[m] = fact[m - 1] * m;
                for (int i = 0; i < need; ++i) {
                    double pw = 1.0;
                    for (int m = 0; m < n; ++m) {
                        A[i * 9 + m] = pw / fact[m];
                        pw *= (double)cand[i];
                    }
                }
                for (int jr = 0; jr <= Pd / 2; ++jr) {
                    const int j = 2 * jr, row = need + jr;
                    for (int m = 0; m < n; ++m) {
                        if (m < j) {
                            A[row * 9 + m] = 0.0;
                        } else {
                            double pw = 1.0;
                            for (int e = 0; e < m - j; ++e) pw *= ub;
                            A[row * 9 + m] = pw / fact[m - j];
                        }
                    }
                }
                if (!small_inverse(A, Ai, n)) {
                    bad = true;
                    continue;
                }
                for (int k = kb; k <= H; ++k) {
                    if (!((ext >> k) & 1u)) continue;
                    // e_i = sum_m phi_m(k) Ai[m][i]
                    for (int i = 0; i < need; ++i) {
                        double e = 0.0, pw = 1.0;
                        for (int m = 0; m < n; ++m) {
                            e += pw / fact[m] * Ai[m * 9 + i];
                            pw *= (double)k;
                        }
                        int o[3] = {0, 0, 0};
                        o[a] = sg * cand[i];
                        const int32_t c = pack_off(o[0], o[1], o[2]);
                        int slot = -1;
                        for (int t = 0; t < ne; ++t)
                            if (code[t] == c) slot = t;
                        if (slot < 0 && ne < FIT1D_MAXE) {
                            slot = ne++;
                            code[slot] = c;
                            wsum[slot] = 0.0;
                        }
                        if (slot >= 0) wsum[slot] += P.w2[H + k] * e;
                    }
                }
            }
        const int64_t st = r * FIT1D_MAXE;
        P.start[r] = st;
        P.cnt[r] = ne;
        for (int t = 0; t < ne; ++t) {
            P.pool_code[st + t] = code[t];
            P.pool_field[st + t] = 0;
            P.pool_w[st + t] = wsum[t];
        }
        P.info[4 * r + 0] = 0;
        P.info[4 * r + 1] = pmin;
        P.info[4 * r + 2] = 0;
        P.info[4 * r + 3] = bad ? 1 : 0;
    }
}

static ib_status run_fit1d(ib_table* t, const Geo& g, const FitKind& fk, int M, const std::vector<double>& w2,
                           cudaStream_t s, DevBuf& tmp) {
    const Layout& L = t->L;
    uint8_t* flags = nullptr;
    TRY(tmp.alloc(&flags, L.N));
    k_row_flags<<<grid_for(L.N, 256), 256, 0, s>>>(g, fk.rule, flags);
    IB_CHECK_LAUNCH("k_row_flags");
    ib_count_launch("setup");
    int64_t* rows = nullptr;
    int64_t nrows = 0;
    TRY(compact(flags, L.N, &rows, &nrows, s));
    tmp.ptrs.push_back(rows);
    Fit1dParams P;
    memset(&P, 0, sizeof P);
    P.g = g;
    P.M = M;
    P.eta = fk.feta[0];
    for (int k = 0; k <= M && k < 9; ++k) P.w2[k] = w2[k];
    P.rows = rows;
    P.nrows = nrows;
    const int64_t nr = std::max<int64_t>(nrows, 1);
    TRY(tmp.alloc(&P.info, 4 * nr));
    TRY(tmp.alloc(&P.cnt, nr));
    TRY(tmp.alloc(&P.start, nr));
    TRY(tmp.alloc(&P.pool_code, nr * FIT1D_MAXE));
    TRY(tmp.alloc(&P.pool_field, nr * FIT1D_MAXE));
    TRY(tmp.alloc(&P.pool_w, nr * FIT1D_MAXE));
    if (nrows) {
        k_fit1d<<<grid_for(nrows, 128), 128, 0, s>>>(P);
        IB_CHECK_LAUNCH("k_fit1d");
        ib_count_launch("setup");
    }
    std::vector<int32_t> hinfo(4 * nrows);
    if (nrows) IB_CUDA(cudaMemcpy(hinfo.data(), P.info, 16 * nrows, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < nrows; ++i) {
        if (hinfo[4 * i + 3] != 0) t->n_fail++;
        else if (hinfo[4 * i + 1] != M) t->n_reduced++;
    }
    return pack_pool(t, fk, rows, nrows, P.info, P.cnt, P.start, P.pool_code, P.pool_field, P.pool_w, 0, s, tmp);
}

static void free_op(IbOp& op) {
    void* ps[] = {op.row_lin, op.row_pad, op.row_ptr, op.col_code, op.col_pad, op.w64, op.w32, op.row_info,
                  op.t_row_pad, op.t_ptr, op.t_src_off, op.t_w64, op.t_w32, op.code16};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (auto& b : op.bins) ib_free_bins(b);
    for (auto& b : op.t_bins) ib_free_bins(b);
    op = IbOp();
}

extern "C" void ib_table_free(ib_table* t) {
    if (!t) return;
    for (int i = 0; i < IB_MAX_OPS; ++i) free_op(t->ops[i]);
    for (int f = 0; f < 4; ++f)
        if (t->mask_pad[f]) cudaFree(t->mask_pad[f]);
    if (t->learned_resid) cudaFree(t->learned_resid);
    delete t;
}

static ib_status build_impl(const ib_grid* grid, const double* sdf, ib_bc bc, ib_form form, const ib_opts* opts_in,
                            ib_mlp* mlp, double accept_tol, ib_table** out, cudaStream_t s) {
    double t0 = ib_wall_seconds();
    if (!grid || !sdf || !out) {
        ib_set_error("null argument");
        return IB_ERR_ARG;
    }
    *out = nullptr;
    int d = grid->ndim;
    if (d != 2 && d != 3) {
        ib_set_error("ndim must be 2 or 3");
        return IB_ERR_ARG;
    }
    for (int a = 0; a < d; ++a)
        if (grid->n[a] < 2 || grid->n[a] > (1 << 20)) {
            ib_set_error("grid size out of range");
            return IB_ERR_ARG;
        }
    if (!(grid->h > 0.0)) {
        ib_set_error("h must be positive");
        return IB_ERR_ARG;
    }
    ib_opts o;
    if (opts_in) o = *opts_in;
    else ib_opts_default(&o, 4);
    int M = o.space_order;
    if (M < 2 || M > 8 || (M & 1)) {
        ib_set_error("space_order must be 2, 4, 6 or 8");
        return IB_ERR_ARG;
    }
    // basis order min(M, 4): the order-reduction paragraph's reduced basis at M > 4
    if (o.basis_order <= 0) o.basis_order = std::min(M, 4);
    if (o.basis_order > M || (o.basis_order & 1)) {
        ib_set_error("basis_order must be even and <= space_order");
        return IB_ERR_ARG;
    }
    if (o.min_order < 2 || o.min_order > o.basis_order) o.min_order = std::min(2, o.basis_order);
    if (!(o.growth >= 0.0) || o.growth > 8.0) o.growth = 3.0;
    // rank tolerance by boundary condition (the paper gives none): the measured
    // growth of the schemes is lowest at 1e-3 for the free surface, 1e-2 for the rigid
    if (!(o.rank_tol > 0.0)) o.rank_tol = bc == IB_RIGID ? 1e-2 : 1e-3;
    // pressure cut-off: the paper's 0.5 for the free surface; 0.25 for the rigid
    // surface, for which the paper gives none (0.5 leaves a growing mode there)
    if (o.eta_p < 0.0) o.eta_p = bc == IB_RIGID ? 0.25 : 0.5;
    if (bc != IB_FREE && bc != IB_RIGID) {
        ib_set_error("bc must be IB_FREE or IB_RIGID");
        return IB_ERR_ARG;
    }
    if (o.extrapolation != IB_EXTRAP_ND && o.extrapolation != IB_EXTRAP_1D) {
        ib_set_error("extrapolation must be IB_EXTRAP_ND or IB_EXTRAP_1D");
        return IB_ERR_ARG;
    }
    if (o.extrapolation == IB_EXTRAP_1D && (form != IB_SECOND_ORDER || bc != IB_FREE || mlp)) {
        ib_set_error("the 1D extrapolation is stated for the free surface of the second-order form");
        return IB_ERR_ARG;
    }
    if (form != IB_SECOND_ORDER && form != IB_FIRST_ORDER_STAGGERED) {
        ib_set_error("unknown form");
        return IB_ERR_ARG;
    }
    ib_table* t = new ib_table();
    t->grid = *grid;
    t->form = form;
    t->bc = bc;
    t->opts = o;
    int64_t n3[3] = {grid->n[0], grid->n[1], d == 3 ? grid->n[2] : 1};
    t->L = make_layout(d, grid->n, std::max(M / 2, 1));
    Geo g;
    g.ndim = d;
    g.n[0] = n3[0];
    g.n[1] = n3[1];
    g.n[2] = n3[2];
    g.sdf = sdf;
    g.inv_h = 1.0 / grid->h;
    // central first-derivative weights for the SDF gradient
    double cf[5][9];
    memset(cf, 0, sizeof cf);
    for (int q = 2; q <= 8; q += 2) {
        std::vector<double> w = central_first(q);
        for (int k = 0; k <= q; ++k) cf[q / 2][k] = w[k];
    }
    ib_status st = IB_OK;
    auto fail = [&](ib_status e) {
        ib_table_free(t);
        return e;
    };
    if (cudaMemcpyToSymbol(c_cfirst, cf, sizeof cf) != cudaSuccess) return fail(IB_ERR_CUDA);
    DevBuf tmp;
    // ---- boundary points
    uint8_t* flags;
    if ((st = tmp.alloc(&flags, t->L.N)) != IB_OK) return fail(st);
    k_bp_flags<<<grid_for(t->L.N, 256), 256, 0, s>>>(g, M, flags);
    if (cudaGetLastError() != cudaSuccess) return fail(IB_ERR_CUDA);
    int64_t* bplist = nullptr;
    int64_t nbp = 0;
    if ((st = compact(flags, t->L.N, &bplist, &nbp, s)) != IB_OK) return fail(st);
    tmp.ptrs.push_back(bplist);
    int32_t* bp_index;
    double *bp_xb, *bp_n;
    if ((st = tmp.alloc(&bp_index, t->L.N)) != IB_OK) return fail(st);
    if ((st = tmp.alloc(&bp_xb, 3 * std::max<int64_t>(nbp, 1))) != IB_OK) return fail(st);
    if ((st = tmp.alloc(&bp_n, 3 * std::max<int64_t>(nbp, 1))) != IB_OK) return fail(st);
    if (cudaMemsetAsync(bp_index, 0xff, sizeof(int32_t) * t->L.N, s) != cudaSuccess) return fail(IB_ERR_CUDA);
    if (nbp) k_bp_write<<<grid_for(nbp, 256), 256, 0, s>>>(g, M, bplist, nbp, bp_index, bp_xb, bp_n);
    if (cudaGetLastError() != cudaSuccess) return fail(IB_ERR_CUDA);
    t->n_bp = nbp;
    // ---- interior masks (padded) used by the propagators
    int nmask = form == IB_SECOND_ORDER ? 1 : 1 + d;
    for (int f = 0; f < nmask; ++f) {
        if (cudaMalloc(&t->mask_pad[f], t->L.total) != cudaSuccess) return fail(IB_ERR_OOM);
        cudaMemsetAsync(t->mask_pad[f], 0, t->L.total, s);
    }
    k_masks<<<grid_for(t->L.N, 256), 256, 0, s>>>(g, t->L, nmask, t->mask_pad[0], t->mask_pad[1], t->mask_pad[2],
                                                  t->mask_pad[3]);
    if (cudaGetLastError() != cudaSuccess) return fail(IB_ERR_CUDA);
    // ---- fits
    const int H = M / 2;
    if (form == IB_SECOND_ORDER) {
        std::vector<double> w2 = ib_central_second(M);
        FitKind fk;
        memset(&fk, 0, sizeof fk);
        fk.rule.row_field = 0;
        int ne = 0;
        for (int a = 0; a < d; ++a)
            for (int k = -H; k <= H; ++k) {
                if (k == 0) continue;
                fk.rule.Efield[ne] = 0;
                fk.rule.Eoff[ne][0] = fk.rule.Eoff[ne][1] = fk.rule.Eoff[ne][2] = 0;
                fk.rule.Eoff[ne][a] = k;
                fk.rule.Ew[ne] = w2[k + H];
                ++ne;
            }
        fk.rule.nE = ne;
        fk.nf = 1;
        fk.fkind[0] = 0;
        fk.feta[0] = o.eta_p;
        fk.vector_bc = false;
        fk.mlp = mlp;
        fk.grid = grid;
        fk.sdf = sdf;
        fk.accept_tol = accept_tol;
        t->nops = 1;
        if (o.extrapolation == IB_EXTRAP_1D)
            st = run_fit1d(t, g, fk, M, w2, s, tmp);
        else
            st = run_fit(t, g, fk, bp_index, bp_xb, bp_n, 0, s, tmp);
        if (st != IB_OK) return fail(st);
    } else {
        std::vector<double> c1 = ib_staggered_first(M);
        t->nops = 2 * d;
        // gradients at v_a nodes: p at j + k e_a, k = -H+1..H, weight c1[k + H - 1]
        for (int a = 0; a < d; ++a) {
            FitKind fk;
            memset(&fk, 0, sizeof fk);
            fk.rule.row_field = 1 + a;
            int ne = 0;
            for (int k = -H + 1; k <= H; ++k) {
                fk.rule.Efield[ne] = 0;
                fk.rule.Eoff[ne][0] = fk.rule.Eoff[ne][1] = fk.rule.Eoff[ne][2] = 0;
                fk.rule.Eoff[ne][a] = k;
                fk.rule.Ew[ne] = c1[k + H - 1];
                ++ne;
            }
            fk.rule.nE = ne;
            fk.nf = 1;
            fk.fkind[0] = 0;
            fk.feta[0] = o.eta_p;
            fk.x0shift2[a] = 1;
            fk.vector_bc = false;
            if ((st = run_fit(t, g, fk, bp_index, bp_xb, bp_n, a, s, tmp)) != IB_OK) return fail(st);
        }
        // divergence at p nodes: v_a at j + k e_a, k = -H..H-1, weight c1[k + H]
        FitKind fk;
        memset(&fk, 0, sizeof fk);
        fk.rule.row_field = 0;
        int ne = 0;
        for (int a = 0; a < d; ++a)
            for (int k = -H; k <= H - 1; ++k) {
                fk.rule.Efield[ne] = 1 + a;
                fk.rule.Eoff[ne][0] = fk.rule.Eoff[ne][1] = fk.rule.Eoff[ne][2] = 0;
                fk.rule.Eoff[ne][a] = k;
                fk.rule.Ew[ne] = c1[k + H];
                ++ne;
            }
        fk.rule.nE = ne;
        fk.nf = d;
        for (int a = 0; a < d; ++a) {
            fk.fkind[a] = 1 + a;
            fk.fshift2[a][a] = 1;
            fk.feta[a] = o.eta_v;
        }
        fk.vector_bc = true;
        if ((st = run_fit(t, g, fk, bp_index, bp_xb, bp_n, d, s, tmp)) != IB_OK) return fail(st);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(IB_ERR_CUDA);
    t->setup_seconds = ib_wall_seconds() - t0;
    *out = t;
    if (t->n_fail) {
        char buf[160];
        snprintf(buf, sizeof buf, "%lld rows could not be constrained", (long long)t->n_fail);
        ib_set_error(buf);
        return IB_ERR_RANK;
    }
    return IB_OK;
}

extern "C" ib_status ib_build_stencils(const ib_grid* grid, const double* sdf_dev, ib_bc bc, ib_form form,
                                       const ib_opts* opts, ib_table** out, void* stream) {
    ib_set_error("");
    return build_impl(grid, sdf_dev, bc, form, opts, nullptr, -1.0, out, (cudaStream_t)stream);
}

extern "C" ib_status ib_build_stencils_learned(const ib_grid* grid, const double* sdf_dev, ib_bc bc,
                                               const ib_opts* opts, ib_mlp* mlp, double accept_tol,
                                               ib_table** out, void* stream) {
    ib_set_error("");
    if (!mlp) {
        ib_set_error("null network");
        return IB_ERR_ARG;
    }
    if (!grid || grid->ndim != ib_mlp_ndim(mlp) || !opts || opts->space_order != ib_mlp_order(mlp)) {
        ib_set_error("the network was configured for another dimension or space order");
        return IB_ERR_ARG;
    }
    return build_impl(grid, sdf_dev, bc, IB_SECOND_ORDER, opts, mlp, accept_tol, out, (cudaStream_t)stream);
}

extern "C" ib_status ib_table_learned(const ib_table* t, int64_t* n_checked, int64_t* n_accepted,
                                      double* resid_host) {
    if (!t) {
        ib_set_error("null table");
        return IB_ERR_ARG;
    }
    if (n_checked) *n_checked = t->learned_checked;
    if (n_accepted) *n_accepted = t->learned_accepted;
    if (resid_host && t->nops > 0) {
        const int64_t n = t->ops[0].nrows;
        if (t->learned_resid) {
            IB_CUDA(cudaMemcpy(resid_host, t->learned_resid, 8 * n, cudaMemcpyDeviceToHost));
        } else {
            for (int64_t i = 0; i < n; ++i) resid_host[i] = NAN;
        }
    }
    return IB_OK;
}

extern "C" ib_status ib_table_stats(const ib_table* t, ib_table_info* info) {
    if (!t || !info) {
        ib_set_error("null argument");
        return IB_ERR_ARG;
    }
    memset(info, 0, sizeof *info);
    info->n_ops = t->nops;
    info->ndim = t->grid.ndim;
    for (int i = 0; i < t->nops; ++i) {
        info->rows[i] = t->ops[i].nrows;
        info->nnz[i] = t->ops[i].nnz;
    }
    info->n_boundary_points = t->n_bp;
    info->n_rank_failures = t->n_fail;
    info->n_grown = t->n_grown;
    info->n_reduced = t->n_reduced;
    info->table_bytes = t->table_bytes;
    info->setup_seconds = t->setup_seconds;
    return IB_OK;
}

extern "C" ib_status ib_table_export(const ib_table* t, int32_t op, int64_t* row_node, int64_t* row_ptr,
                                     int32_t* col_off, double* weight, int32_t* row_info) {
    if (!t || op < 0 || op >= t->nops) {
        ib_set_error("bad table or operator index");
        return IB_ERR_ARG;
    }
    const IbOp& o = t->ops[op];
    if (row_node && o.nrows) IB_CUDA(cudaMemcpy(row_node, o.row_lin, 8 * o.nrows, cudaMemcpyDeviceToHost));
    if (row_ptr) IB_CUDA(cudaMemcpy(row_ptr, o.row_ptr, 8 * (o.nrows + 1), cudaMemcpyDeviceToHost));
    if (row_info && o.nrows) IB_CUDA(cudaMemcpy(row_info, o.row_info, 16 * o.nrows, cudaMemcpyDeviceToHost));
    if (weight && o.nnz) IB_CUDA(cudaMemcpy(weight, o.w64, 8 * o.nnz, cudaMemcpyDeviceToHost));
    if (col_off && o.nnz) {
        std::vector<int32_t> codes(o.nnz);
        IB_CUDA(cudaMemcpy(codes.data(), o.col_code, 4 * o.nnz, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < o.nnz; ++i) {
            int dx, dy, dz;
            unpack_off(codes[i], dx, dy, dz);
            // logical (x, y, z) with the 2D second axis stored in slot 1 (= z)
            if (t->grid.ndim == 2) {
                col_off[3 * i + 0] = dx;
                col_off[3 * i + 1] = 0;
                col_off[3 * i + 2] = dy;
            } else {
                col_off[3 * i + 0] = dx;
                col_off[3 * i + 1] = dy;
                col_off[3 * i + 2] = dz;
            }
        }
    }
    return IB_OK;
}

// ---------------------------------------------------------------------------
// tile binning of IB rows (used by the fused step kernels)
// ---------------------------------------------------------------------------
__global__ void k_tile_keys(int64_t n, const int64_t* pad, Layout L, int tx, int ty, int tz, int64_t ntx,
                            int64_t nty, int32_t* keys, int32_t* vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = pad[i] - L.base;
        int64_t z = q / L.plane;
        int64_t rem = q - z * L.plane;
        int64_t y = rem / L.px;
        int64_t x = rem - y * L.px;
        if (L.ndim == 2) y = 0;
        int64_t key = ((z / tz) * nty + (y / ty)) * ntx + (x / tx);
        keys[i] = (int32_t)key;
        vals[i] = (int32_t)i;
    }
}

__global__ void k_tile_ptr(int64_t n, const int32_t* sorted_keys, int64_t ntiles, int32_t* ptr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t kprev = i == 0 ? -1 : sorted_keys[i - 1];
        int32_t kcur = i == n ? (int32_t)ntiles : sorted_keys[i];
        for (int32_t k = kprev + 1; k <= kcur; ++k) ptr[k] = (int32_t)i;
    }
}

__global__ void k_perm_nnz(int64_t n, const int32_t* perm, const int64_t* row_ptr, int64_t* cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = perm[k];
        cnt[k] = row_ptr[r + 1] - row_ptr[r];
    }
}

__global__ void k_ent_ptr(int64_t ntiles, const int32_t* tile_ptr, const int64_t* ent_off, int32_t* ent_ptr) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= ntiles; t += (int64_t)gridDim.x * blockDim.x)
        ent_ptr[t] = (int32_t)ent_off[tile_ptr[t]];
}

// one block per row (in tile order): expand its entries relative to the tile origin
__global__ void k_fill_entries(int64_t n, const int32_t* perm, const int32_t* sorted_keys, const int64_t* ent_off,
                               const int64_t* row_pad, const int64_t* row_ptr, const int64_t* col_pad,
                               const double* w64, Layout L, TileBins b, int32_t* loc, int32_t* src, float* w32o,
                               double* w64o) {
    for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
        const int32_t r = perm[k];
        const int64_t org = tile_origin(L, b, sorted_keys[k]);
        const int64_t q = row_pad[r];
        const int64_t rel = q - org;
        int32_t lx, ly;
        if (L.ndim == 2) {
            int64_t dz = rel >= 0 ? rel / L.px : -((-rel + L.px - 1) / L.px);
            ly = (int32_t)dz;
            lx = (int32_t)(rel - dz * L.px);
        } else {
            int64_t dy = rel / L.px;
            ly = (int32_t)dy;
            lx = (int32_t)(rel - dy * L.px);
        }
        const int32_t lidx = ly * b.tx + lx;
        const int64_t o = ent_off[k];
        const int64_t j0 = row_ptr[r];
        for (int64_t j = j0 + threadIdx.x; j < row_ptr[r + 1]; j += blockDim.x) {
            loc[o + (j - j0)] = lidx;
            src[o + (j - j0)] = (int32_t)(rel + col_pad[j]);
            w32o[o + (j - j0)] = (float)w64[j];
            w64o[o + (j - j0)] = w64[j];
        }
    }
}

void ib_free_bins(TileBins& b) {
    void* ps[] = {b.tile_ptr, b.perm, b.ent_ptr, b.ent_loc, b.ent_src, b.ent_w32, b.ent_w64,
                  b.ent_code, b.ent_slot};
    for (void* p : ps)
        if (p) cudaFree(p);
    b = TileBins();
}

// compact entries: 16-bit footprint code (and one-byte slot) per entry
__global__ void k_fill_compact(int64_t n, const int32_t* perm, const int32_t* ent_loc, const int64_t* ent_off,
                               const int64_t* row_ptr, const int32_t* col_code, uint16_t* ent_code,
                               uint8_t* ent_slot) {
    for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
        const int32_t r = perm[k];
        const int64_t o = ent_off[k];
        const int64_t j0 = row_ptr[r], j1 = row_ptr[r + 1];
        for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            int dx, dy, dz;
            unpack_off(col_code[j], dx, dy, dz);
            ent_code[o + (j - j0)] = pack_code16(dx, dy, dz);
            if (ent_slot) ent_slot[o + (j - j0)] = (uint8_t)ent_loc[o];
        }
    }
}

// rows (row_pad) binned by tile; with row_ptr/col_pad/w64 also the flattened entries
// (and, with col_code, their compact form)
static ib_status make_bins(const Layout& L, int64_t n, const int64_t* pad, const int64_t* row_ptr,
                           const int64_t* col_pad, const double* w64, int tx, int ty, int tz, TileBins& b,
                           cudaStream_t s, const int32_t* col_code = nullptr) {
    int64_t ntx = (L.nx + tx - 1) / tx;
    int64_t nty = (L.ny + ty - 1) / ty;
    int64_t ntz = (L.nz + tz - 1) / tz;
    b.tx = tx;
    b.ty = ty;
    b.tz = tz;
    b.ntx = ntx;
    b.nty = nty;
    b.ntiles = ntx * nty * ntz;
    TRY(dalloc(&b.tile_ptr, b.ntiles + 1));
    TRY(dalloc(&b.perm, std::max<int64_t>(n, 1)));
    TRY(dalloc(&b.ent_ptr, b.ntiles + 1));
    if (n == 0) {
        IB_CUDA(cudaMemsetAsync(b.tile_ptr, 0, sizeof(int32_t) * (b.ntiles + 1), s));
        IB_CUDA(cudaMemsetAsync(b.ent_ptr, 0, sizeof(int32_t) * (b.ntiles + 1), s));
        TRY(dalloc(&b.ent_loc, 1));
        TRY(dalloc(&b.ent_src, 1));
        TRY(dalloc(&b.ent_w32, 1));
        TRY(dalloc(&b.ent_w64, 1));
        IB_CUDA(cudaStreamSynchronize(s));
        return IB_OK;
    }
    DevBuf tmp;
    int32_t *keys, *vals, *keys2;
    TRY(tmp.alloc(&keys, n));
    TRY(tmp.alloc(&vals, n));
    TRY(tmp.alloc(&keys2, n));
    k_tile_keys<<<grid_for(n, 256), 256, 0, s>>>(n, pad, L, tx, ty, tz, ntx, nty, keys, vals);
    IB_CHECK_LAUNCH("k_tile_keys");
    ib_count_launch("setup");
    size_t tb = 0;
    IB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, keys, keys2, vals, b.perm, (int)n, 0, 32, s));
    void* dt;
    IB_CUDA(cudaMalloc(&dt, tb + 16));
    tmp.ptrs.push_back(dt);
    IB_CUDA(cub::DeviceRadixSort::SortPairs(dt, tb, keys, keys2, vals, b.perm, (int)n, 0, 32, s));
    k_tile_ptr<<<grid_for(n + 1, 256), 256, 0, s>>>(n, keys2, b.ntiles, b.tile_ptr);
    IB_CHECK_LAUNCH("k_tile_ptr");
    ib_count_launch("setup");
    if (row_ptr) {
        int64_t *cnt, *off;
        TRY(tmp.alloc(&cnt, n + 1));
        TRY(tmp.alloc(&off, n + 1));
        IB_CUDA(cudaMemsetAsync(cnt + n, 0, sizeof(int64_t), s));
        k_perm_nnz<<<grid_for(n, 256), 256, 0, s>>>(n, b.perm, row_ptr, cnt);
        IB_CHECK_LAUNCH("k_perm_nnz");
        TRY(excl_scan(cnt, off, n + 1, s));
        IB_CUDA(cudaMemcpy(&b.nent, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (b.nent >= (int64_t)1 << 31) {
            ib_set_error("correction table too large for 32-bit tile entry offsets");
            return IB_ERR_ARG;
        }
        TRY(dalloc(&b.ent_loc, std::max<int64_t>(b.nent, 1)));
        TRY(dalloc(&b.ent_src, std::max<int64_t>(b.nent, 1)));
        TRY(dalloc(&b.ent_w32, std::max<int64_t>(b.nent, 1)));
        TRY(dalloc(&b.ent_w64, std::max<int64_t>(b.nent, 1)));
        k_ent_ptr<<<grid_for(b.ntiles + 1, 256), 256, 0, s>>>(b.ntiles, b.tile_ptr, off, b.ent_ptr);
        k_fill_entries<<<grid_for(n, 1), 64, 0, s>>>(n, b.perm, keys2, off, pad, row_ptr, col_pad, w64, L, b,
                                                     b.ent_loc, b.ent_src, b.ent_w32, b.ent_w64);
        IB_CHECK_LAUNCH("k_fill_entries");
        ib_count_launch("setup");
        if (col_code) {
            TRY(dalloc(&b.ent_code, std::max<int64_t>(b.nent, 1)));
            if ((int64_t)tx * ty * tz <= 256) TRY(dalloc(&b.ent_slot, std::max<int64_t>(b.nent, 1)));
            k_fill_compact<<<grid_for(n, 1), 64, 0, s>>>(n, b.perm, b.ent_loc, off, row_ptr, col_code, b.ent_code,
                                                         b.ent_slot);
            IB_CHECK_LAUNCH("k_fill_compact");
            ib_count_launch("setup");
        }
    } else {
        IB_CUDA(cudaMemsetAsync(b.ent_ptr, 0, sizeof(int32_t) * (b.ntiles + 1), s));
    }
    IB_CUDA(cudaStreamSynchronize(s));
    return IB_OK;
}

__global__ void k_code16(int64_t nnz, const int32_t* col_code, uint16_t* out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x) {
        int dx, dy, dz;
        unpack_off(col_code[j], dx, dy, dz);
        out[j] = pack_code16(dx, dy, dz);
    }
}

// 16-bit footprint codes of an operator's entries in row order (kept with the table)
ib_status ib_table_code16(ib_table* t, int op, const uint16_t** out, cudaStream_t s) {
    IbOp& o = t->ops[op];
    if (!o.code16 && o.nnz > 0) {
        TRY(dalloc(&o.code16, o.nnz));
        k_code16<<<grid_for(o.nnz, 256), 256, 0, s>>>(o.nnz, o.col_code, o.code16);
        IB_CHECK_LAUNCH("k_code16");
        ib_count_launch("setup");
    }
    *out = o.code16;
    return IB_OK;
}

ib_status ib_make_bins_ext(const Layout& L, int64_t n, const int64_t* pad, int tx, int ty, int tz, TileBins& b,
                           cudaStream_t s) {
    return make_bins(L, n, pad, nullptr, nullptr, nullptr, tx, ty, tz, b, s);
}

ib_status ib_table_bins(ib_table* t, int op, bool transposed, int tx, int ty, int tz, const TileBins** out,
                        cudaStream_t s) {
    IbOp& o = t->ops[op];
    std::vector<TileBins>& v = transposed ? o.t_bins : o.bins;
    for (auto& b : v)
        if (b.tx == tx && b.ty == ty && b.tz == tz) {
            *out = &b;
            return IB_OK;
        }
    TileBins b;
    if (transposed) {
        TRY(ib_table_transpose(t, op, s));
        TRY(make_bins(t->L, o.t_nrows, o.t_row_pad, o.t_ptr, o.t_src_off, o.t_w64, tx, ty, tz, b, s));
    } else {
        TRY(make_bins(t->L, o.nrows, o.row_pad, o.row_ptr, o.col_pad, o.w64, tx, ty, tz, b, s, o.col_code));
    }
    v.push_back(b);
    *out = &v.back();
    return IB_OK;
}

// ---------------------------------------------------------------------------
// transposed operator: entries (row i, col j = i + off, w) regrouped by j
// ---------------------------------------------------------------------------
__global__ void k_expand_entries(int64_t nrows, const int64_t* row_ptr, const int64_t* row_pad, const int64_t* col_pad,
                                 int64_t* key, int64_t* idx) {
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x)
        for (int64_t k = row_ptr[r] + threadIdx.x; k < row_ptr[r + 1]; k += blockDim.x) {
            key[k] = row_pad[r] + col_pad[k];
            idx[k] = k;
        }
}
__global__ void k_entry_rows(int64_t nrows, const int64_t* row_ptr, int64_t* entry_row) {
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x)
        for (int64_t k = row_ptr[r] + threadIdx.x; k < row_ptr[r + 1]; k += blockDim.x) entry_row[k] = r;
}
__global__ void k_transpose_fill(int64_t nnz, const int64_t* skey, const int64_t* sidx, const int64_t* entry_row,
                                 const int64_t* row_pad, const double* w64, int64_t* src_off, double* tw64,
                                 float* tw32, uint8_t* head) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = sidx[k];
        int64_t j = skey[k];
        src_off[k] = row_pad[entry_row[e]] - j;
        tw64[k] = w64[e];
        tw32[k] = (float)w64[e];
        head[k] = (k == 0 || skey[k - 1] != j) ? 1 : 0;
    }
}
__global__ void k_transpose_rows(int64_t nheads, const int64_t* head_pos, const int64_t* skey, int64_t nnz,
                                 int64_t* t_row_pad, int64_t* t_ptr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nheads; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nheads) {
            t_ptr[i] = head_pos[i];
            t_row_pad[i] = skey[head_pos[i]];
        } else {
            t_ptr[i] = nnz;
        }
    }
}

ib_status ib_table_transpose(ib_table* t, int op, cudaStream_t s) {
    IbOp& o = t->ops[op];
    if (o.have_t) return IB_OK;
    int64_t nnz = o.nnz;
    DevBuf tmp;
    if (nnz == 0) {
        o.t_nrows = 0;
        TRY(dalloc(&o.t_ptr, 1));
        IB_CUDA(cudaMemset(o.t_ptr, 0, 8));
        TRY(dalloc(&o.t_row_pad, 1));
        TRY(dalloc(&o.t_src_off, 1));
        TRY(dalloc(&o.t_w64, 1));
        TRY(dalloc(&o.t_w32, 1));
        o.have_t = true;
        return IB_OK;
    }
    int64_t *key, *idx, *skey, *sidx, *erow;
    TRY(tmp.alloc(&key, nnz));
    TRY(tmp.alloc(&idx, nnz));
    TRY(tmp.alloc(&skey, nnz));
    TRY(tmp.alloc(&sidx, nnz));
    TRY(tmp.alloc(&erow, nnz));
    k_expand_entries<<<grid_for(o.nrows, 1), 64, 0, s>>>(o.nrows, o.row_ptr, o.row_pad, o.col_pad, key, idx);
    k_entry_rows<<<grid_for(o.nrows, 1), 64, 0, s>>>(o.nrows, o.row_ptr, erow);
    IB_CHECK_LAUNCH("k_expand_entries");
            ib_count_launch("setup");
    size_t tb = 0;
    IB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, key, skey, idx, sidx, (int)nnz, 0, 64, s));
    void* dt;
    IB_CUDA(cudaMalloc(&dt, tb + 16));
    tmp.ptrs.push_back(dt);
    IB_CUDA(cub::DeviceRadixSort::SortPairs(dt, tb, key, skey, idx, sidx, (int)nnz, 0, 64, s));
    uint8_t* head;
    TRY(tmp.alloc(&head, nnz));
    TRY(dalloc(&o.t_src_off, nnz));
    TRY(dalloc(&o.t_w64, nnz));
    TRY(dalloc(&o.t_w32, nnz));
    k_transpose_fill<<<grid_for(nnz, 256), 256, 0, s>>>(nnz, skey, sidx, erow, o.row_pad, o.w64, o.t_src_off, o.t_w64,
                                                        o.t_w32, head);
    IB_CHECK_LAUNCH("k_transpose_fill");
            ib_count_launch("setup");
    int64_t* heads;
    int64_t nheads = 0;
    TRY(compact(head, nnz, &heads, &nheads, s));
    tmp.ptrs.push_back(heads);
    TRY(dalloc(&o.t_row_pad, nheads));
    TRY(dalloc(&o.t_ptr, nheads + 1));
    k_transpose_rows<<<grid_for(nheads + 1, 256), 256, 0, s>>>(nheads, heads, skey, nnz, o.t_row_pad, o.t_ptr);
    IB_CHECK_LAUNCH("k_transpose_rows");
            ib_count_launch("setup");
    IB_CUDA(cudaStreamSynchronize(s));
    o.t_nrows = nheads;
    o.have_t = true;
    return IB_OK;
}
