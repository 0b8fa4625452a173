// Learned modified stencils: input features, a bfloat16 tensor-core MLP
// (mma.sync m16n8k16, FP32 accumulation), its training step (mean squared
// error, Adam) and the row predictions that the constructor checks.
//
// The paper fits every modified row by constrained least squares; the network
// only proposes rows, and ib_build_stencils_learned keeps a proposal when it
// passes the exactness test of the fit (see k_fit's learned_residual).
#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "ib_common.cuh"

#define TRY(x)                                  \
    do {                                        \
        ib_status st_ = (x);                    \
        if (st_ != IB_OK) return st_;           \
    } while (0)

#define MLP_MAX_LINEAR 9
typedef __nv_bfloat16 bf16;

struct ib_mlp {
    int device = 0;
    ib_mlp_config cfg;
    int nl = 0;                         // linear layers
    int dims[MLP_MAX_LINEAR + 1];       // dims[0] = n_in, dims[nl] = n_out
    int64_t w_off[MLP_MAX_LINEAR], b_off[MLP_MAX_LINEAR], wb_off[MLP_MAX_LINEAR];
    int64_t n_params = 0, n_wb = 0;
    int n_in_off = 0, n_in = 0, n_out = 0, out_R = 0;
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    bf16* wb = nullptr;                 // bfloat16 copies of the weight matrices
    int8_t* in_off = nullptr;           // [n_in_off][3]
    int32_t* out_lut = nullptr;         // [(2R+1)^3] footprint index or -1
    int64_t step = 0;
    // training scratch (rows <= cap)
    int64_t cap = 0;
    bf16* act = nullptr;                // hidden activations, [nl - 1][cap][n_hidden]
    float* y = nullptr;                 // [cap][n_out]
    float* g32 = nullptr;               // [cap][max dim]
    bf16* g16a = nullptr;
    bf16* g16b = nullptr;
    float* part = nullptr;              // [1024] loss partial sums
    // inference scratch (rows per chunk)
    int64_t icap = 0;
    bf16* ia = nullptr;
    bf16* ib = nullptr;
    bf16* ix = nullptr;                 // features of one chunk
};

// ---------------------------------------------------------------------------
// offsets |o| <= r in support order: distance, then array order (z, y, x)
// ---------------------------------------------------------------------------
static std::vector<std::array<int, 3>> ball_offsets(int d, double r) {
    const int R = (int)std::ceil(r) + 1;
    const int64_t q_lim = (int64_t)std::floor(4.0 * r * r + 1e-9);
    struct E {
        int64_t q;
        int z, y, x;
    };
    std::vector<E> e;
    for (int z = (d == 3 ? -R : 0); z <= (d == 3 ? R : 0); ++z)
        for (int y = -R; y <= R; ++y)
            for (int x = -R; x <= R; ++x) {
                int64_t q = 4LL * (x * x + y * y + z * z);
                if (q <= q_lim) e.push_back({q, z, y, x});
            }
    std::sort(e.begin(), e.end(), [](const E& a, const E& b) {
        if (a.q != b.q) return a.q < b.q;
        if (a.z != b.z) return a.z < b.z;
        if (a.y != b.y) return a.y < b.y;
        return a.x < b.x;
    });
    std::vector<std::array<int, 3>> out;
    // in 2D the second coordinate is the array's second axis: (x, y) with z = 0
    for (auto& v : e) out.push_back({v.x, v.y, v.z});
    return out;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__global__ void k_features(int ndim, int64_t n0, int64_t n1, int64_t n2, double h, const double* sdf,
                           const int64_t* nodes, int64_t n, const int8_t* off, int noff, int n_in,
                           float f_free, float f_rigid, float f_order, bf16* X) {
    const int64_t total = n * n_in;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n_in;
        const int j = (int)(e - i * n_in);
        float v;
        if (j < noff) {
            const int64_t lin = nodes[i];
            int64_t x = lin % n0, r = lin / n0, y, z;
            if (ndim == 3) {
                y = r % n1;
                z = r / n1;
            } else {
                y = r;
                z = 0;
            }
            int64_t qx = x + off[3 * j], qy = y + off[3 * j + 1], qz = z + off[3 * j + 2];
            qx = qx < 0 ? 0 : (qx >= n0 ? n0 - 1 : qx);
            qy = qy < 0 ? 0 : (qy >= n1 ? n1 - 1 : qy);
            qz = qz < 0 ? 0 : (qz >= n2 ? n2 - 1 : qz);
            v = (float)(sdf[(qz * n1 + qy) * n0 + qx] / h);
        } else if (j == noff) {
            v = f_free;
        } else if (j == noff + 1) {
            v = f_rigid;
        } else {
            v = f_order;
        }
        X[e] = __float2bfloat16(v);
    }
}

// C = A B with bfloat16 operands and FP32 accumulation on the tensor cores.
//   A(m, k) = A[row_a(m) * a_sm + k * a_sk], row_a(m) = a_idx ? a_idx[m] : m
//   B(k, n) = B[row_b(k) * b_sk + n * b_sn], row_b(k) = b_idx ? b_idx[k] : k
enum { EPI_BIAS_F32 = 0, EPI_BIAS_RELU_BF16 = 1, EPI_RELU_GRAD = 2, EPI_F32 = 3 };
struct Gemm {
    int M, N, K;
    const bf16* A;
    int64_t a_sm, a_sk;
    const int64_t* a_idx;
    const bf16* B;
    int64_t b_sk, b_sn;
    const int64_t* b_idx;
    int mode;
    const float* bias;      // [N]
    const bf16* act;        // EPI_RELU_GRAD: forward activation [m][n] (ld act_ld); gradient kept where > 0
    int64_t act_ld;
    float* c32;
    bf16* c16;
    int64_t ldc;
};

#define GBM 64
#define GBN 64
#define GBK 32
#define GLD (GBK + 8)

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_16816(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm(Gemm g) {
    __shared__ __align__(16) bf16 As[GBM * GLD];
    __shared__ __align__(16) bf16 Bs[GBN * GLD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gr = lane >> 2, tc = (lane & 3) * 2;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const bool a_kfast = g.a_sk == 1, b_kfast = g.b_sk == 1;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < g.K; k0 += GBK) {
        for (int e = tid; e < GBM * GBK; e += 128) {
            int r, kk;
            if (a_kfast) {
                r = e / GBK;
                kk = e - r * GBK;
            } else {
                kk = e / GBM;
                r = e - kk * GBM;
            }
            const int m = m0 + r, k = k0 + kk;
            bf16 v = zero;
            if (m < g.M && k < g.K) {
                const int64_t row = g.a_idx ? g.a_idx[m] : (int64_t)m;
                v = g.A[row * g.a_sm + (int64_t)k * g.a_sk];
            }
            As[r * GLD + kk] = v;
        }
        for (int e = tid; e < GBN * GBK; e += 128) {
            int c, kk;
            if (b_kfast) {
                c = e / GBK;
                kk = e - c * GBK;
            } else {
                kk = e / GBN;
                c = e - kk * GBN;
            }
            const int n = n0 + c, k = k0 + kk;
            bf16 v = zero;
            if (n < g.N && k < g.K) {
                const int64_t kr = g.b_idx ? g.b_idx[k] : (int64_t)k;
                v = g.B[kr * g.b_sk + (int64_t)n * g.b_sn];
            }
            Bs[c * GLD + kk] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const bf16* p = As + (wm + i * 16 + gr) * GLD + ks + tc;
                af[i][0] = ld_pair(p);
                af[i][1] = ld_pair(p + 8 * GLD);
                af[i][2] = ld_pair(p + 8);
                af[i][3] = ld_pair(p + 8 * GLD + 8);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bf16* p = Bs + (wn + j * 8 + gr) * GLD + ks + tc;
                bfr[j][0] = ld_pair(p);
                bfr[j][1] = ld_pair(p + 8);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + i * 16 + gr + (e >> 1) * 8;
                const int n = n0 + wn + j * 8 + tc + (e & 1);
                if (m >= g.M || n >= g.N) continue;
                const float x = acc[i][j][e];
                const int64_t q = (int64_t)m * g.ldc + n;
                if (g.mode == EPI_BIAS_F32) {
                    g.c32[q] = x + g.bias[n];
                } else if (g.mode == EPI_BIAS_RELU_BF16) {
                    g.c16[q] = __float2bfloat16(fmaxf(x + g.bias[n], 0.f));
                } else if (g.mode == EPI_RELU_GRAD) {
                    const float keep = __bfloat162float(g.act[(int64_t)m * g.act_ld + n]) > 0.f ? x : 0.f;
                    g.c32[q] = keep;
                    g.c16[q] = __float2bfloat16(keep);
                } else {
                    g.c32[q] = x;
                }
            }
}

// dY = 2 (Y - T[idx]) / (n n_out) (FP32 and bfloat16), per-block partial sums of (Y - T)^2
__global__ void k_mse_grad(const float* Y, const float* T, const int64_t* idx, int64_t n, int no, float scale,
                           float* g32, bf16* g16, float* part) {
    __shared__ float red[8];
    float acc = 0.f;
    const int64_t total = n * no;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / no;
        const int j = (int)(e - i * no);
        const float d = Y[e] - T[idx[i] * no + j];
        acc += d * d;
        const float gv = scale * d;
        g32[e] = gv;
        g16[e] = __float2bfloat16(gv);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_loss_final(const float* part, int nb, float inv, float* loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nb; ++i) t += part[i];
        *loss = (float)(t * inv);
    }
}

// db[n] = sum_m G[m][n]; block (32, 8) per 32 columns
__global__ void k_colsum(const float* G, int64_t M, int N, float* out) {
    __shared__ float red[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    float a = 0.f;
    if (n < N)
        for (int64_t m = threadIdx.y; m < M; m += 8) a += G[m * N + n];
    red[threadIdx.y][threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.f;
        for (int r = 0; r < 8; ++r) t += red[r][threadIdx.x];
        out[n] = t;
    }
}

// Adam (Kingma & Ba, Algorithm 1); bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
__global__ void k_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

struct WeightCopy {
    int nl;
    int64_t w_off[MLP_MAX_LINEAR], wb_off[MLP_MAX_LINEAR], cnt[MLP_MAX_LINEAR];
};
__global__ void k_sync_weights(WeightCopy c, const float* p, bf16* wb) {
    const int l = blockIdx.y;
    if (l >= c.nl) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.cnt[l]; i += (int64_t)gridDim.x * blockDim.x)
        wb[c.wb_off[l] + i] = __float2bfloat16(p[c.w_off[l] + i]);
}

// training targets of the Laplacian rows of a plain table
__global__ void k_target_flags(int64_t nrows, const int32_t* info, const int64_t* row_ptr, const int32_t* code,
                               const int32_t* lut, int R, int r2, int order, uint8_t* flags) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        bool ok = info[4 * r + 3] == 0 && info[4 * r + 0] == r2 && info[4 * r + 1] == order;
        const int W = 2 * R + 1;
        for (int64_t e = row_ptr[r]; ok && e < row_ptr[r + 1]; ++e) {
            int dx, dy, dz;
            unpack_off(code[e], dx, dy, dz);
            if (dx < -R || dx > R || dy < -R || dy > R || dz < -R || dz > R ||
                lut[((dz + R) * W + (dy + R)) * W + (dx + R)] < 0)
                ok = false;
        }
        flags[r] = ok ? 1 : 0;
    }
}

__global__ void k_target_write(int64_t n, const int64_t* sel, const int64_t* row_lin, const int64_t* row_ptr,
                               const int32_t* code, const double* w, const int32_t* lut, int R, int no,
                               int64_t* nodes, float* T) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = sel[k];
        nodes[k] = row_lin[r];
        float* t = T + k * no;
        for (int j = 0; j < no; ++j) t[j] = 0.f;
        const int W = 2 * R + 1;
        // a Laplacian row holds each support node once
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            int dx, dy, dz;
            unpack_off(code[e], dx, dy, dz);
            t[lut[((dz + R) * W + (dy + R)) * W + (dx + R)]] = (float)w[e];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int grid1(int64_t n, int bs) {
    int64_t b = (n + bs - 1) / bs;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

template <class T>
static ib_status mlp_alloc(T** p, int64_t n) {
    *p = nullptr;
    if (n <= 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)n);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        ib_set_error("device allocation failed in the learned-stencil network");
        return IB_ERR_OOM;
    }
    return IB_OK;
}

static ib_status launch_gemm(const Gemm& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return IB_OK;
    dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM);
    if (grid.y > 65535) {
        ib_set_error("GEMM too tall");
        return IB_ERR_ARG;
    }
    k_gemm<<<grid, 128, 0, s>>>(g);
    IB_CHECK_LAUNCH("k_gemm");
    ib_count_launch("mlp_gemm_bf16");
    return IB_OK;
}

static Gemm gemm_fwd(const ib_mlp* m, int l, const bf16* Xin, int64_t ldx, const int64_t* idx, int64_t n) {
    Gemm g;
    memset(&g, 0, sizeof g);
    g.M = (int)n;
    g.N = m->dims[l + 1];
    g.K = m->dims[l];
    g.A = Xin;
    g.a_sm = ldx;
    g.a_sk = 1;
    g.a_idx = idx;
    g.B = m->wb + m->wb_off[l];   // W_l [N][K]: B(k, n) = W[n][k]
    g.b_sk = 1;
    g.b_sn = g.K;
    g.bias = m->params + m->b_off[l];
    return g;
}

extern "C" ib_status ib_mlp_create(const ib_mlp_config* cfg, ib_mlp** out) {
    ib_set_error("");
    if (!cfg || !out) {
        ib_set_error("null argument");
        return IB_ERR_ARG;
    }
    *out = nullptr;
    if ((cfg->ndim != 2 && cfg->ndim != 3) || cfg->space_order < 2 || cfg->space_order > 8 ||
        (cfg->space_order & 1) || cfg->n_hidden < 8 || cfg->n_hidden > 1024 || (cfg->n_hidden & 7) ||
        cfg->n_layers < 1 || cfg->n_layers > MLP_MAX_LINEAR - 1 || !(cfg->in_radius >= 0.0) ||
        cfg->in_radius > 8.0 || !(cfg->out_radius > 0.0) || cfg->out_radius > 8.0) {
        ib_set_error("ib_mlp_config out of range");
        return IB_ERR_ARG;
    }
    ib_mlp* m = new ib_mlp();
    m->cfg = *cfg;
    cudaGetDevice(&m->device);
    auto fail = [&](ib_status st) {
        ib_mlp_free(m);
        return st;
    };
    auto inb = ball_offsets(cfg->ndim, cfg->in_radius);
    auto outb = ball_offsets(cfg->ndim, cfg->out_radius);
    m->n_in_off = (int)inb.size();
    m->n_in = m->n_in_off + 3;
    m->n_out = (int)outb.size();
    m->out_R = (int)std::ceil(cfg->out_radius);
    m->nl = cfg->n_layers + 1;
    m->dims[0] = m->n_in;
    for (int l = 1; l < m->nl; ++l) m->dims[l] = cfg->n_hidden;
    m->dims[m->nl] = m->n_out;
    int64_t p = 0, wb = 0;
    for (int l = 0; l < m->nl; ++l) {
        m->w_off[l] = p;
        p += (int64_t)m->dims[l + 1] * m->dims[l];
        m->b_off[l] = p;
        p += m->dims[l + 1];
        m->wb_off[l] = wb;
        wb += (int64_t)m->dims[l + 1] * m->dims[l];
        wb = (wb + 7) & ~(int64_t)7;   // 16-byte aligned matrices
    }
    m->n_params = p;
    m->n_wb = wb;
    ib_status st;
    if ((st = mlp_alloc(&m->params, p)) != IB_OK) return fail(st);
    if ((st = mlp_alloc(&m->grads, p)) != IB_OK) return fail(st);
    if ((st = mlp_alloc(&m->adam_m, p)) != IB_OK) return fail(st);
    if ((st = mlp_alloc(&m->adam_v, p)) != IB_OK) return fail(st);
    if ((st = mlp_alloc(&m->wb, wb)) != IB_OK) return fail(st);
    if ((st = mlp_alloc(&m->in_off, 3 * (int64_t)inb.size())) != IB_OK) return fail(st);
    const int W = 2 * m->out_R + 1;
    if ((st = mlp_alloc(&m->out_lut, (int64_t)W * W * W)) != IB_OK) return fail(st);
    if ((st = mlp_alloc(&m->part, 1024)) != IB_OK) return fail(st);
    std::vector<int8_t> ho;
    for (auto& o : inb)
        for (int a = 0; a < 3; ++a) ho.push_back((int8_t)o[a]);
    std::vector<int32_t> lut((size_t)W * W * W, -1);
    for (size_t j = 0; j < outb.size(); ++j) {
        const auto& o = outb[j];
        lut[((size_t)(o[2] + m->out_R) * W + (o[1] + m->out_R)) * W + (o[0] + m->out_R)] = (int32_t)j;
    }
    if (cudaMemcpy(m->in_off, ho.data(), ho.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->out_lut, lut.data(), lut.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->params, 0, 4 * p) != cudaSuccess || cudaMemset(m->grads, 0, 4 * p) != cudaSuccess ||
        cudaMemset(m->adam_m, 0, 4 * p) != cudaSuccess || cudaMemset(m->adam_v, 0, 4 * p) != cudaSuccess ||
        cudaMemset(m->wb, 0, 2 * wb) != cudaSuccess) {
        ib_set_error("initialising the network failed");
        return fail(IB_ERR_CUDA);
    }
    *out = m;
    return IB_OK;
}

extern "C" void ib_mlp_free(ib_mlp* m) {
    if (!m) return;
    void* ptrs[] = {m->params, m->grads, m->adam_m, m->adam_v, m->wb, m->in_off, m->out_lut, m->act,
                    m->y, m->g32, m->g16a, m->g16b, m->part, m->ia, m->ib, m->ix};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete m;
}

extern "C" ib_status ib_mlp_info(const ib_mlp* m, int64_t* n_in, int64_t* n_out, int64_t* n_params) {
    if (!m) {
        ib_set_error("null network");
        return IB_ERR_ARG;
    }
    if (n_in) *n_in = m->n_in;
    if (n_out) *n_out = m->n_out;
    if (n_params) *n_params = m->n_params;
    return IB_OK;
}

extern "C" ib_status ib_mlp_buffers(ib_mlp* m, float** params, float** grads, float** am, float** av) {
    if (!m) {
        ib_set_error("null network");
        return IB_ERR_ARG;
    }
    if (params) *params = m->params;
    if (grads) *grads = m->grads;
    if (am) *am = m->adam_m;
    if (av) *av = m->adam_v;
    return IB_OK;
}

static ib_status sync_weights(ib_mlp* m, cudaStream_t s) {
    WeightCopy c;
    memset(&c, 0, sizeof c);
    c.nl = m->nl;
    int64_t mx = 0;
    for (int l = 0; l < m->nl; ++l) {
        c.w_off[l] = m->w_off[l];
        c.wb_off[l] = m->wb_off[l];
        c.cnt[l] = (int64_t)m->dims[l + 1] * m->dims[l];
        mx = std::max(mx, c.cnt[l]);
    }
    dim3 grid(grid1(mx, 256), m->nl);
    k_sync_weights<<<grid, 256, 0, s>>>(c, m->params, m->wb);
    IB_CHECK_LAUNCH("k_sync_weights");
    ib_count_launch("mlp_setup");
    return IB_OK;
}

extern "C" ib_status ib_mlp_sync_weights(ib_mlp* m, void* stream) {
    if (!m) {
        ib_set_error("null network");
        return IB_ERR_ARG;
    }
    return sync_weights(m, (cudaStream_t)stream);
}

static ib_status features(const ib_mlp* m, const ib_grid* grid, const double* sdf, const int64_t* nodes,
                          int64_t n, ib_bc bc, bf16* X, cudaStream_t s) {
    if (!grid || !sdf || (n > 0 && (!nodes || !X))) {
        ib_set_error("null argument");
        return IB_ERR_ARG;
    }
    if (grid->ndim != m->cfg.ndim) {
        ib_set_error("grid dimension differs from the network's");
        return IB_ERR_ARG;
    }
    if (n <= 0) return IB_OK;
    const int64_t n2 = grid->ndim == 3 ? grid->n[2] : 1;
    k_features<<<grid1(n * m->n_in, 256), 256, 0, s>>>(
        grid->ndim, grid->n[0], grid->n[1], n2, grid->h, sdf, nodes, n, m->in_off, m->n_in_off, m->n_in,
        bc == IB_FREE ? 1.f : 0.f, bc == IB_RIGID ? 1.f : 0.f, (float)(m->cfg.space_order / 8.0), X);
    IB_CHECK_LAUNCH("k_features");
    ib_count_launch("mlp_features");
    return IB_OK;
}

extern "C" ib_status ib_mlp_features(const ib_mlp* m, const ib_grid* grid, const double* sdf_dev,
                                     const int64_t* nodes_dev, int64_t n, ib_bc bc, void* X_dev, void* stream) {
    ib_set_error("");
    if (!m) {
        ib_set_error("null network");
        return IB_ERR_ARG;
    }
    return features(m, grid, sdf_dev, nodes_dev, n, bc, (bf16*)X_dev, (cudaStream_t)stream);
}

static const int64_t kChunk = 1 << 16;

static ib_status ensure_infer(ib_mlp* m) {
    if (m->icap >= kChunk) return IB_OK;
    TRY(mlp_alloc(&m->ia, kChunk * m->cfg.n_hidden));
    TRY(mlp_alloc(&m->ib, kChunk * m->cfg.n_hidden));
    TRY(mlp_alloc(&m->ix, kChunk * m->n_in));
    m->icap = kChunk;
    return IB_OK;
}

// Y[n][n_out] = network(X[n][n_in]) in chunks of kChunk rows
static ib_status forward(ib_mlp* m, const bf16* X, int64_t n, float* Y, cudaStream_t s) {
    TRY(ensure_infer(m));
    const int H = m->cfg.n_hidden;
    for (int64_t c0 = 0; c0 < n; c0 += kChunk) {
        const int64_t cn = std::min(kChunk, n - c0);
        const bf16* in = X + c0 * m->n_in;
        int64_t ldi = m->n_in;
        bf16* bufs[2] = {m->ia, m->ib};
        for (int l = 0; l < m->nl; ++l) {
            Gemm g = gemm_fwd(m, l, in, ldi, nullptr, cn);
            if (l + 1 < m->nl) {
                g.mode = EPI_BIAS_RELU_BF16;
                g.c16 = bufs[l & 1];
                g.ldc = H;
                TRY(launch_gemm(g, s));
                in = bufs[l & 1];
                ldi = H;
            } else {
                g.mode = EPI_BIAS_F32;
                g.c32 = Y + c0 * m->n_out;
                g.ldc = m->n_out;
                TRY(launch_gemm(g, s));
            }
        }
    }
    return IB_OK;
}

extern "C" ib_status ib_mlp_forward(ib_mlp* m, const void* X_dev, int64_t n, float* Y_dev, void* stream) {
    ib_set_error("");
    if (!m || (n > 0 && (!X_dev || !Y_dev)) || n < 0) {
        ib_set_error("null argument");
        return IB_ERR_ARG;
    }
    return forward(m, (const bf16*)X_dev, n, Y_dev, (cudaStream_t)stream);
}

static ib_status ensure_train(ib_mlp* m, int64_t n) {
    if (n <= m->cap) return IB_OK;
    const int H = m->cfg.n_hidden;
    int mxd = 0;
    for (int l = 0; l <= m->nl; ++l) mxd = std::max(mxd, m->dims[l]);
    void* ptrs[] = {m->act, m->y, m->g32, m->g16a, m->g16b};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    m->act = nullptr;
    m->y = nullptr;
    m->g32 = nullptr;
    m->g16a = m->g16b = nullptr;
    m->cap = 0;
    TRY(mlp_alloc(&m->act, (int64_t)(m->nl - 1) * n * H));
    TRY(mlp_alloc(&m->y, n * m->n_out));
    TRY(mlp_alloc(&m->g32, n * mxd));
    TRY(mlp_alloc(&m->g16a, n * mxd));
    TRY(mlp_alloc(&m->g16b, n * mxd));
    m->cap = n;
    return IB_OK;
}

extern "C" ib_status ib_mlp_train_step(ib_mlp* m, const void* X_dev, const float* T_dev, const int64_t* idx_dev,
                                       int64_t n, float lr, float beta1, float beta2, float eps, float* loss_dev,
                                       void* stream) {
    ib_set_error("");
    cudaStream_t s = (cudaStream_t)stream;
    if (!m || !X_dev || !T_dev || !idx_dev || !loss_dev || n <= 0 || n > (1 << 22)) {
        ib_set_error("bad argument (rows must be 1 .. 4194304)");
        return IB_ERR_ARG;
    }
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f)) {
        ib_set_error("bad Adam hyper-parameters");
        return IB_ERR_ARG;
    }
    TRY(ensure_train(m, n));
    const int H = m->cfg.n_hidden, L = m->nl;
    const bf16* X = (const bf16*)X_dev;
    auto act = [&](int l) { return m->act + (int64_t)(l - 1) * m->cap * H; };   // input of layer l >= 1
    // forward, keeping each layer's input
    for (int l = 0; l < L; ++l) {
        Gemm g = l == 0 ? gemm_fwd(m, 0, X, m->n_in, idx_dev, n) : gemm_fwd(m, l, act(l), H, nullptr, n);
        if (l + 1 < L) {
            g.mode = EPI_BIAS_RELU_BF16;
            g.c16 = act(l + 1);
            g.ldc = H;
        } else {
            g.mode = EPI_BIAS_F32;
            g.c32 = m->y;
            g.ldc = m->n_out;
        }
        TRY(launch_gemm(g, s));
    }
    // loss and output gradient
    const int nb = std::min(1024, grid1(n * m->n_out, 256));
    k_mse_grad<<<nb, 256, 0, s>>>(m->y, T_dev, idx_dev, n, m->n_out, (float)(2.0 / ((double)n * m->n_out)), m->g32,
                                  m->g16a, m->part);
    IB_CHECK_LAUNCH("k_mse_grad");
    ib_count_launch("mlp_loss");
    k_loss_final<<<1, 32, 0, s>>>(m->part, nb, (float)(1.0 / ((double)n * m->n_out)), loss_dev);
    IB_CHECK_LAUNCH("k_loss_final");
    ib_count_launch("mlp_loss");
    // backward: g16 holds d loss / d (output of layer l), g32 its FP32 value
    bf16* gcur = m->g16a;
    bf16* gnext = m->g16b;
    for (int l = L - 1; l >= 0; --l) {
        const int No = m->dims[l + 1], Ki = m->dims[l];
        // dW_l [No][Ki] = G^T X_l
        Gemm gw;
        memset(&gw, 0, sizeof gw);
        gw.M = No;
        gw.N = Ki;
        gw.K = (int)n;
        gw.A = gcur;          // A(o, r) = G[r][o]
        gw.a_sm = 1;
        gw.a_sk = No;
        if (l == 0) {
            gw.B = X;         // B(r, k) = X[idx[r]][k]
            gw.b_sk = m->n_in;
            gw.b_idx = idx_dev;
        } else {
            gw.B = act(l);
            gw.b_sk = H;
        }
        gw.b_sn = 1;
        gw.mode = EPI_F32;
        gw.c32 = m->grads + m->w_off[l];
        gw.ldc = Ki;
        TRY(launch_gemm(gw, s));
        // db_l = column sums of G (FP32)
        k_colsum<<<(No + 31) / 32, dim3(32, 8), 0, s>>>(m->g32, n, No, m->grads + m->b_off[l]);
        IB_CHECK_LAUNCH("k_colsum");
        ib_count_launch("mlp_colsum");
        if (l > 0) {
            // G_{l-1} = (G W_l) * [X_l > 0]
            Gemm gx;
            memset(&gx, 0, sizeof gx);
            gx.M = (int)n;
            gx.N = Ki;
            gx.K = No;
            gx.A = gcur;
            gx.a_sm = No;
            gx.a_sk = 1;
            gx.B = m->wb + m->wb_off[l];   // B(o, k) = W[o][k]
            gx.b_sk = Ki;
            gx.b_sn = 1;
            gx.mode = EPI_RELU_GRAD;
            gx.act = act(l);
            gx.act_ld = H;
            gx.c32 = m->g32;
            gx.c16 = gnext;
            gx.ldc = Ki;
            TRY(launch_gemm(gx, s));
            std::swap(gcur, gnext);
        }
    }
    // Adam
    m->step += 1;
    const double bc1 = 1.0 - std::pow((double)beta1, (double)m->step);
    const double bc2 = 1.0 - std::pow((double)beta2, (double)m->step);
    k_adam<<<grid1(m->n_params, 256), 256, 0, s>>>(m->n_params, m->params, m->grads, m->adam_m, m->adam_v, lr, beta1,
                                                   beta2, eps, (float)bc1, (float)bc2);
    IB_CHECK_LAUNCH("k_adam");
    ib_count_launch("mlp_adam");
    return sync_weights(m, s);
}

extern "C" ib_status ib_mlp_targets(const ib_table* t, const ib_mlp* m, int64_t* nodes_dev, float* T_dev,
                                    int64_t cap, int64_t* n_rows, void* stream) {
    ib_set_error("");
    cudaStream_t s = (cudaStream_t)stream;
    if (!t || !m || !n_rows || (cap > 0 && (!nodes_dev || !T_dev))) {
        ib_set_error("null argument");
        return IB_ERR_ARG;
    }
    if (t->form != IB_SECOND_ORDER || t->grid.ndim != m->cfg.ndim) {
        ib_set_error("targets need a second-order table of the network's dimension");
        return IB_ERR_ARG;
    }
    const IbOp& op = t->ops[0];
    *n_rows = 0;
    if (op.nrows == 0) return IB_OK;
    uint8_t* flags = nullptr;
    TRY(mlp_alloc(&flags, op.nrows));
    const int r2 = (int)lrint(2.0 * m->cfg.out_radius);
    k_target_flags<<<grid1(op.nrows, 256), 256, 0, s>>>(op.nrows, op.row_info, op.row_ptr, op.col_code, m->out_lut,
                                                         m->out_R, r2, t->opts.basis_order, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(flags);
        return ib_cuda_fail(e, "k_target_flags", __FILE__, __LINE__);
    }
    ib_count_launch("mlp_targets");
    int64_t* sel = nullptr;
    int64_t cnt = 0;
    ib_status st = ib_compact(flags, op.nrows, &sel, &cnt, s);
    cudaFree(flags);
    if (st != IB_OK) return st;
    const int64_t n = std::min(cnt, cap);
    if (n > 0) {
        k_target_write<<<grid1(n, 128), 128, 0, s>>>(n, sel, op.row_lin, op.row_ptr, op.col_code, op.w64, m->out_lut,
                                                      m->out_R, m->n_out, nodes_dev, T_dev);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaFree(sel);
            return ib_cuda_fail(e, "k_target_write", __FILE__, __LINE__);
        }
        ib_count_launch("mlp_targets");
    }
    e = cudaStreamSynchronize(s);
    cudaFree(sel);
    if (e != cudaSuccess) return ib_cuda_fail(e, "ib_mlp_targets", __FILE__, __LINE__);
    *n_rows = n;
    return IB_OK;
}

// ---------------------------------------------------------------------------
// internal interface of the constructor
// ---------------------------------------------------------------------------
int ib_mlp_out_count(const ib_mlp* m) { return m->n_out; }
double ib_mlp_out_radius(const ib_mlp* m) { return m->cfg.out_radius; }
int ib_mlp_ndim(const ib_mlp* m) { return m->cfg.ndim; }
int ib_mlp_order(const ib_mlp* m) { return m->cfg.space_order; }
const int32_t* ib_mlp_lut(const ib_mlp* m, int* R) {
    *R = m->out_R;
    return m->out_lut;
}

ib_status ib_mlp_predict_nodes(ib_mlp* m, const ib_grid* grid, const double* sdf, const int64_t* nodes, int64_t n,
                               ib_bc bc, float* Y, cudaStream_t s) {
    TRY(ensure_infer(m));
    for (int64_t c0 = 0; c0 < n; c0 += kChunk) {
        const int64_t cn = std::min(kChunk, n - c0);
        TRY(features(m, grid, sdf, nodes + c0, cn, bc, m->ix, s));
        TRY(forward(m, m->ix, cn, Y + c0 * m->n_out, s));
    }
    return IB_OK;
}
