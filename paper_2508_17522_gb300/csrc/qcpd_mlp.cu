// The learned form (warm start and diagonal preconditioner for the Krylov
// solve): per-row features of a plan, a 16-256-256-2 MLP with BF16 weights
// and FP32 accumulation on the tensor cores (forward, backward, Adam), the
// decoding of its outputs into (warm start, preconditioner), and the export
// of a solve's embedding-space solution that the training targets come from.
//
// The GEMMs use the warp-level mma.sync m16n8k16 BF16 instruction: the MLP
// is under 1% of a learned solve's time (a few GFLOP per training step),
// so it is written for clarity and exact agreement with its CPU check rather
// than for tcgen05 throughput.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qcpd_kernels.cuh"
#include "qcpd_plan.h"

namespace qcpd {

constexpr int kIn = QCP_MLP_IN, kHid = QCP_MLP_HIDDEN, kOut = QCP_MLP_OUT;
// packed parameter layout: W1 [kHid x kIn], b1 [kHid], W2 [kHid x kHid], b2 [kHid], W3 [kOut x kHid], b3 [kOut]
constexpr int64_t kW1 = 0, kB1 = kW1 + kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + (int64_t)kHid * kHid,
                  kW3 = kB2 + kHid, kB3 = kW3 + kOut * kHid, kNParam = kB3 + kOut;

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------- GEMM
// C(m, n) (+)= sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn], C(m, n) = C[m ldc + n]; BF16 inputs, FP32 sums.
struct GemmArgs {
    const bf16* A;
    int64_t sam, sak;
    const bf16* B;
    int64_t sbk, sbn;
    float* C;
    int64_t ldc;
    int M, N, K, accumulate;
};

constexpr int GBM = 64, GBN = 64, GBK = 32;

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 64 x 64 tile per CTA, 4 warps of 32 x 32 (2 x 4 MMA tiles of 16 x 8).
__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
    __shared__ __align__(16) bf16 As[GBM][GBK + 8];
    __shared__ __align__(16) bf16 Bs[GBN][GBK + 8];
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gr = lane >> 2, tc = (lane & 3) * 2;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < g.K; k0 += GBK) {
        for (int i = tid; i < GBM * GBK; i += 128) {
            const int mm = i / GBK, kk = i % GBK, m = m0 + mm, k = k0 + kk;
            As[mm][kk] = (m < g.M && k < g.K) ? g.A[m * g.sam + k * g.sak] : zero;
        }
        for (int i = tid; i < GBN * GBK; i += 128) {
            const int nn = i / GBK, kk = i % GBK, n = n0 + nn, k = k0 + kk;
            Bs[nn][kk] = (n < g.N && k < g.K) ? g.B[k * g.sbk + n * g.sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm + mi * 16 + gr;
                a[mi][0] = ld_pair(&As[r][ks + tc]);
                a[mi][1] = ld_pair(&As[r + 8][ks + tc]);
                a[mi][2] = ld_pair(&As[r][ks + tc + 8]);
                a[mi][3] = ld_pair(&As[r + 8][ks + tc + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int c = wn + ni * 8 + gr;
                b[ni][0] = ld_pair(&Bs[c][ks + tc]);
                b[ni][1] = ld_pair(&Bs[c][ks + tc + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = m0 + wm + mi * 16 + gr + (e >= 2 ? 8 : 0);
                const int c = n0 + wn + ni * 8 + tc + (e & 1);
                if (r < g.M && c < g.N) {
                    float* p = g.C + (int64_t)r * g.ldc + c;
                    *p = g.accumulate ? *p + acc[mi][ni][e] : acc[mi][ni][e];
                }
            }
}

static void gemm(cudaStream_t st, const bf16* A, int64_t sam, int64_t sak, const bf16* B, int64_t sbk, int64_t sbn,
                 float* C, int64_t ldc, int M, int N, int K) {
    GemmArgs g{A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, 0};
    dim3 grid((unsigned)((N + GBN - 1) / GBN), (unsigned)((M + GBM - 1) / GBM));
    k_gemm_bf16<<<grid, 128, 0, st>>>(g);
}

// ---------------------------------------------------------------- elementwise
__global__ void k_to_bf16(const float* in, int64_t n, bf16* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// x' = (x - mean) * inv_std per feature, then BF16
__global__ void k_norm_bf16(const float* x, int64_t rows, const float* mean, const float* inv_std, bf16* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * kIn) return;
    const int f = (int)(i % kIn);
    out[i] = __float2bfloat16_rn((x[i] - mean[f]) * inv_std[f]);
}

// pre += bias (per column); h = relu(pre) as BF16
__global__ void k_bias_relu(float* pre, const float* bias, int64_t rows, int cols, bf16* h) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const float v = pre[i] + bias[i % cols];
    pre[i] = v;
    h[i] = __float2bfloat16_rn(v > 0.f ? v : 0.f);
}

__global__ void k_bias(float* y, const float* bias, int64_t rows, int cols) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < rows * cols) y[i] += bias[i % cols];
}

// Per block: sum of w (y - t)^2 and of w over its rows (fixed order).
__global__ void k_loss_part(const float* y, const float* t, const float* w, int64_t n, double* part) {
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double d = (double)y[i] - (double)t[i];
        a += (double)w[i] * d * d;
        b += (double)w[i];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

// loss = sum w (y - t)^2 / max(sum w, 1); dy = 2 w (y - t) / max(sum w, 1)
__global__ void k_loss_grad(const float* y, const float* t, const float* w, int64_t n, const double* part, int nparts,
                            float* dy, double* loss) {
    __shared__ double tot[2];
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < nparts; ++k) {
            a += part[2 * k];
            b += part[2 * k + 1];
        }
        tot[0] = a;
        tot[1] = b > 1.0 ? b : 1.0;
        if (blockIdx.x == 0) *loss = a / tot[1];
    }
    __syncthreads();
    const float scale = (float)(2.0 / tot[1]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dy[i] = scale * w[i] * (y[i] - t[i]);
}

// dh[r][j] = (sum_k dy[r][k] W3[k][j]) [pre2[r][j] > 0], FP32 and BF16
__global__ void k_back3(const float* dy, const bf16* W3b, const float* pre2, int64_t rows, float* dh, bf16* dhb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * kHid) return;
    const int64_t r = i / kHid;
    const int j = (int)(i % kHid);
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < kOut; ++k) v = fmaf(dy[r * kOut + k], __bfloat162float(W3b[k * kHid + j]), v);
    v = pre2[i] > 0.f ? v : 0.f;
    dh[i] = v;
    dhb[i] = __float2bfloat16_rn(v);
}

// dh = dh * [pre > 0] in place, and its BF16 copy
__global__ void k_relu_back(float* dh, const float* pre, int64_t n, bf16* dhb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = pre[i] > 0.f ? dh[i] : 0.f;
    dh[i] = v;
    dhb[i] = __float2bfloat16_rn(v);
}

// Column sums out[j] = sum_r a[r][j] (and, with b, out[k][j] = sum_r a[r][k] b[r][j]
// for the last layer's weights), in fixed order: 1024-row chunks, then chunks.
constexpr int kChunkRows = 1024;
__global__ void k_colsum_part(const float* a, int64_t rows, int cols, float* part) {
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    const int64_t r0 = (int64_t)blockIdx.x * kChunkRows, r1 = (rows < r0 + kChunkRows) ? rows : r0 + kChunkRows;
    float s = 0.f;
    for (int64_t r = r0; r < r1; ++r) s += a[r * cols + j];
    part[(int64_t)blockIdx.x * cols + j] = s;
}

__global__ void k_w3_part(const float* dy, const bf16* h2b, int64_t rows, float* part) {
    const int j = threadIdx.x;  // kHid threads
    const int64_t r0 = (int64_t)blockIdx.x * kChunkRows, r1 = (rows < r0 + kChunkRows) ? rows : r0 + kChunkRows;
    float s[kOut] = {};
    for (int64_t r = r0; r < r1; ++r) {
        const float h = __bfloat162float(h2b[r * kHid + j]);
#pragma unroll
        for (int k = 0; k < kOut; ++k) s[k] = fmaf(dy[r * kOut + k], h, s[k]);
    }
#pragma unroll
    for (int k = 0; k < kOut; ++k) part[(int64_t)blockIdx.x * kOut * kHid + k * kHid + j] = s[k];
}

__global__ void k_sum_parts(const float* part, int nparts, int len, float* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    float s = 0.f;
    for (int k = 0; k < nparts; ++k) s += part[(int64_t)k * len + j];
    out[j] = s;
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters, then their BF16 copies.
__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2, bf16* pb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

// v = y + offset; warm_i = scale v_i0, d_i = exp(clamp(v_i1, -8, 8))
__global__ void k_decode(const float* y, const float* offset, int64_t rows, double scale, double* warm, double* d) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    double v0 = (double)y[i * kOut], v1 = (double)y[i * kOut + 1];
    if (offset) {
        v0 += (double)offset[i * kOut];
        v1 += (double)offset[i * kOut + 1];
    }
    if (warm) warm[i] = scale * v0;
    if (d) d[i] = exp(fmin(8.0, fmax(-8.0, v1)));
}

// ---------------------------------------------------------------- features
// Per embedding row (all problems of the plan, in order), QCP_MLP_IN values:
//  0 one; 1-5 row kind (x, zero, R+, SOC, tau); 6 x_i | y_i | 1; 7 z_i = y_i - s_i;
//  8 q_i | b_i; 9 g_i = (2 P x + q)_i | s_i | kappa; 10 diagonal of D Pi (SOC: of the
//  block's D); 11 log ||M row|| / 4; 12 log(nnz(M row) + 1) / 4; 13 SOC block size / 32;
//  14 1 on SOC entries after the block's first; 15 feature 6 times feature 10.
__global__ void k_features(const int64_t* mrowptr, const double* mval_norm2, const double* coefA,
                           const double* coefB, const double* pz, const double* zy, const int8_t* kind,
                           const double* ddiag, const int32_t* socdim, const int8_t* socpos, int64_t Ntot,
                           const int64_t* mrow_of, const double* kappa_of, const int32_t* prob_of, float* out) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= Ntot) return;
    float f[kIn];
    for (int k = 0; k < kIn; ++k) f[k] = 0.f;
    const int kd = kind[r];  // 0 x, 1 zero, 2 R+, 3 SOC, 4 tau
    f[0] = 1.f;
    f[1 + kd] = 1.f;
    const int pi = prob_of[r];
    const int64_t mr = mrow_of[r];
    f[6] = (float)pz[r];
    if (kd >= 1 && kd <= 3) {
        f[7] = (float)zy[r];
        f[9] = (float)(pz[r] - zy[r]);
    }
    if (kd == 0) f[9] = (float)coefB[r];
    if (kd == 4) f[9] = (float)kappa_of[pi];
    f[8] = (float)coefA[r];
    f[10] = (float)ddiag[r];
    const int64_t len = mrowptr[mr + 1] - mrowptr[mr];
    f[11] = len > 0 ? (float)(0.125 * log(mval_norm2[r] + 1e-300)) : 0.f;
    f[12] = (float)(0.25 * log((double)len + 1.0));
    if (kd == 3) {
        f[13] = socdim[r] / 32.f;
        f[14] = (float)socpos[r];
    }
    f[15] = f[6] * f[10];
    for (int k = 0; k < kIn; ++k) out[r * kIn + k] = f[k];
}

template <typename T>
__global__ void k_rownorm2(const int64_t* mrowptr, const T* mval, const int64_t* mrow_of, int64_t Ntot, double* out) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= Ntot) return;
    const int64_t mr = mrow_of[r];
    double s = 0.0;
    for (int64_t k = mrowptr[mr]; k < mrowptr[mr + 1]; ++k) s += (double)mval[k] * (double)mval[k];
    out[r] = s;
}

// the diagonal of D Pi on every row (SOC blocks: the diagonal of the block's
// derivative: 1/2 on the t entry, (t + r - (t/r^2) u_k^2) / (2r) on u_k)
__global__ void k_ddiag(const int8_t* flag, const SocBlock* blocks, int64_t nb, const double* zy, double* dd) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const SocBlock B = blocks[b];
    for (int k = 0; k < B.dim; ++k) {
        double v;
        if (B.kase == 0) v = 0.0;
        else if (B.kase == 1) v = 1.0;
        else if (k == 0) v = 0.5;
        else {
            const double u = zy[B.start + k];
            v = (B.t + B.r - B.tq * u * u) * B.h;
        }
        dd[B.start + k] = v;
    }
}

}  // namespace qcpd

using namespace qcpd;

struct qcp_mlp {
    cudaStream_t stream = nullptr;
    int max_rows = 0;
    int64_t step = 0;
    DevBuf p, g, m, v, pb;                  // FP32 params, grads, Adam moments; BF16 params
    DevBuf xb, pre1, pre2, h1b, h2b, y, dy;  // activations
    DevBuf dh2, dh2b, dh1, dh1b, part, lpart, loss;
    DevBuf norm;  // input mean and 1/std (2 x kIn)
};

extern "C" {

int32_t qcp_mlp_param_count(void) { return (int32_t)kNParam; }

int qcp_mlp_create(int32_t max_rows, void* stream, qcp_mlp** out) {
    if (!out || max_rows < 1) {
        set_error("qcp_mlp_create: max_rows >= 1 and an output pointer required");
        return QCP_ERR_ARG;
    }
    qcp_mlp* q = new qcp_mlp();
    q->stream = static_cast<cudaStream_t>(stream);
    q->max_rows = max_rows;
    const int64_t R = max_rows;
    const int64_t nparts = (R + kChunkRows - 1) / kChunkRows;
    int rc = QCP_OK;
    auto A = [&](DevBuf& b, size_t bytes) {
        if (rc == QCP_OK) rc = b.alloc(bytes);
    };
    A(q->p, 4 * kNParam);
    A(q->g, 4 * kNParam);
    A(q->m, 4 * kNParam);
    A(q->v, 4 * kNParam);
    A(q->pb, 2 * kNParam);
    A(q->xb, 2 * R * kIn);
    A(q->pre1, 4 * R * kHid);
    A(q->pre2, 4 * R * kHid);
    A(q->h1b, 2 * R * kHid);
    A(q->h2b, 2 * R * kHid);
    A(q->y, 4 * R * kOut);
    A(q->dy, 4 * R * kOut);
    A(q->dh2, 4 * R * kHid);
    A(q->dh2b, 2 * R * kHid);
    A(q->dh1, 4 * R * kHid);
    A(q->dh1b, 2 * R * kHid);
    A(q->part, 4 * (size_t)nparts * std::max<int64_t>(kHid * kOut, kHid));
    A(q->lpart, 8 * 2 * 256);
    A(q->loss, 8);
    A(q->norm, 4 * 2 * kIn);
    if (rc != QCP_OK) {
        delete q;
        return rc;
    }
    cudaMemsetAsync(q->p.p, 0, 4 * kNParam, q->stream);
    cudaMemsetAsync(q->m.p, 0, 4 * kNParam, q->stream);
    cudaMemsetAsync(q->v.p, 0, 4 * kNParam, q->stream);
    cudaMemsetAsync(q->pb.p, 0, 2 * kNParam, q->stream);
    float hn[2 * kIn];
    for (int f = 0; f < kIn; ++f) {
        hn[f] = 0.f;
        hn[kIn + f] = 1.f;
    }
    cudaMemcpyAsync(q->norm.p, hn, sizeof(hn), cudaMemcpyHostToDevice, q->stream);
    cudaStreamSynchronize(q->stream);
    *out = q;
    return QCP_OK;
}

int qcp_mlp_set_input_norm(qcp_mlp* q, const float* mean, const float* inv_std) {
    if (!q || !mean || !inv_std) {
        set_error("qcp_mlp_set_input_norm: null argument");
        return QCP_ERR_ARG;
    }
    float hn[2 * kIn];
    std::memcpy(hn, mean, sizeof(float) * kIn);
    std::memcpy(hn + kIn, inv_std, sizeof(float) * kIn);
    QCP_CUDA(cudaMemcpyAsync(q->norm.p, hn, sizeof(hn), cudaMemcpyHostToDevice, q->stream));
    QCP_CUDA(cudaStreamSynchronize(q->stream));
    return QCP_OK;
}

int qcp_mlp_destroy(qcp_mlp* q) {
    if (q) {
        if (q->stream) cudaStreamSynchronize(q->stream);
        delete q;
    }
    return QCP_OK;
}

int qcp_mlp_set_params(qcp_mlp* q, const float* host) {
    if (!q || !host) {
        set_error("qcp_mlp_set_params: null argument");
        return QCP_ERR_ARG;
    }
    QCP_CUDA(cudaMemcpyAsync(q->p.p, host, 4 * kNParam, cudaMemcpyHostToDevice, q->stream));
    QCP_CUDA(cudaMemsetAsync(q->m.p, 0, 4 * kNParam, q->stream));
    QCP_CUDA(cudaMemsetAsync(q->v.p, 0, 4 * kNParam, q->stream));
    q->step = 0;
    k_to_bf16<<<(unsigned)((kNParam + 255) / 256), 256, 0, q->stream>>>(q->p.as<float>(), kNParam, q->pb.as<bf16>());
    QCP_CUDA(cudaGetLastError());
    QCP_CUDA(cudaStreamSynchronize(q->stream));
    return QCP_OK;
}

int qcp_mlp_get_params(const qcp_mlp* q, float* host) {
    if (!q || !host) {
        set_error("qcp_mlp_get_params: null argument");
        return QCP_ERR_ARG;
    }
    QCP_CUDA(cudaMemcpyAsync(host, q->p.p, 4 * kNParam, cudaMemcpyDeviceToHost, q->stream));
    QCP_CUDA(cudaStreamSynchronize(q->stream));
    return QCP_OK;
}

static int mlp_forward(qcp_mlp* q, const float* x, int rows) {
    cudaStream_t st = q->stream;
    const int64_t R = rows;
    const bf16* W = q->pb.as<bf16>();
    const float* P = q->p.as<float>();
    k_norm_bf16<<<(unsigned)((R * kIn + 255) / 256), 256, 0, st>>>(x, R, q->norm.as<float>(),
                                                                  q->norm.as<float>() + kIn, q->xb.as<bf16>());
    // pre1 = x W1^T: A(r, i) = xb[r kIn + i], B(i, j) = W1[j kIn + i]
    gemm(st, q->xb.as<bf16>(), kIn, 1, W + kW1, 1, kIn, q->pre1.as<float>(), kHid, rows, kHid, kIn);
    k_bias_relu<<<(unsigned)((R * kHid + 255) / 256), 256, 0, st>>>(q->pre1.as<float>(), P + kB1, R, kHid,
                                                                   q->h1b.as<bf16>());
    gemm(st, q->h1b.as<bf16>(), kHid, 1, W + kW2, 1, kHid, q->pre2.as<float>(), kHid, rows, kHid, kHid);
    k_bias_relu<<<(unsigned)((R * kHid + 255) / 256), 256, 0, st>>>(q->pre2.as<float>(), P + kB2, R, kHid,
                                                                   q->h2b.as<bf16>());
    gemm(st, q->h2b.as<bf16>(), kHid, 1, W + kW3, 1, kHid, q->y.as<float>(), kOut, rows, kOut, kHid);
    k_bias<<<(unsigned)((R * kOut + 255) / 256), 256, 0, st>>>(q->y.as<float>(), P + kB3, R, kOut);
    QCP_CUDA(cudaGetLastError());
    return QCP_OK;
}

int qcp_mlp_forward(qcp_mlp* q, const float* x, int32_t rows, float* y) {
    if (!q || !x || !y || rows < 0 || rows > q->max_rows) {
        set_error("qcp_mlp_forward: null argument or rows outside [0, max_rows]");
        return QCP_ERR_ARG;
    }
    if (rows == 0) return QCP_OK;
    QCP_TRY(mlp_forward(q, x, rows));
    QCP_CUDA(cudaMemcpyAsync(y, q->y.p, 4 * (size_t)rows * kOut, cudaMemcpyDeviceToDevice, q->stream));
    QCP_CUDA(cudaStreamSynchronize(q->stream));
    return QCP_OK;
}

int qcp_mlp_train_step(qcp_mlp* q, const float* x, const float* target, const float* weight, int32_t rows, float lr,
                       double* loss_host, float* grad_host) {
    if (!q || !x || !target || !weight || rows < 1 || rows > q->max_rows || !(lr >= 0.f)) {
        set_error("qcp_mlp_train_step: null argument, rows outside [1, max_rows] or negative lr");
        return QCP_ERR_ARG;
    }
    cudaStream_t st = q->stream;
    const int64_t R = rows;
    QCP_TRY(mlp_forward(q, x, rows));
    const bf16* W = q->pb.as<bf16>();
    float* G = q->g.as<float>();
    // loss and dy
    const int lp = (int)std::min<int64_t>(256, (R * kOut + 255) / 256);
    k_loss_part<<<lp, 256, 0, st>>>(q->y.as<float>(), target, weight, R * kOut, q->lpart.as<double>());
    k_loss_grad<<<(unsigned)std::min<int64_t>(1024, (R * kOut + 255) / 256), 256, 0, st>>>(
        q->y.as<float>(), target, weight, R * kOut, q->lpart.as<double>(), lp, q->dy.as<float>(), q->loss.as<double>());
    const int64_t nparts = (R + kChunkRows - 1) / kChunkRows;
    float* part = q->part.as<float>();
    // layer 3: dW3 = dy^T h2, db3 = column sums of dy
    k_w3_part<<<(unsigned)nparts, kHid, 0, st>>>(q->dy.as<float>(), q->h2b.as<bf16>(), R, part);
    k_sum_parts<<<(kOut * kHid + 255) / 256, 256, 0, st>>>(part, (int)nparts, kOut * kHid, G + kW3);
    k_colsum_part<<<dim3((unsigned)nparts, 1), 32, 0, st>>>(q->dy.as<float>(), R, kOut, part);
    k_sum_parts<<<1, 32, 0, st>>>(part, (int)nparts, kOut, G + kB3);
    // dh2 = (dy W3) [pre2 > 0]
    k_back3<<<(unsigned)((R * kHid + 255) / 256), 256, 0, st>>>(q->dy.as<float>(), W + kW3, q->pre2.as<float>(), R,
                                                              q->dh2.as<float>(), q->dh2b.as<bf16>());
    // dW2 = dh2^T h1 (tensor cores), db2 = column sums of dh2
    gemm(st, q->dh2b.as<bf16>(), 1, kHid, q->h1b.as<bf16>(), kHid, 1, G + kW2, kHid, kHid, kHid, rows);
    k_colsum_part<<<dim3((unsigned)nparts, kHid / 256), 256, 0, st>>>(q->dh2.as<float>(), R, kHid, part);
    k_sum_parts<<<1, kHid, 0, st>>>(part, (int)nparts, kHid, G + kB2);
    // dh1 = (dh2 W2) [pre1 > 0]: A(r, j) = dh2b[r kHid + j], B(j, i) = W2[j kHid + i]
    gemm(st, q->dh2b.as<bf16>(), kHid, 1, W + kW2, kHid, 1, q->dh1.as<float>(), kHid, rows, kHid, kHid);
    k_relu_back<<<(unsigned)((R * kHid + 255) / 256), 256, 0, st>>>(q->dh1.as<float>(), q->pre1.as<float>(), R * kHid,
                                                                  q->dh1b.as<bf16>());
    // dW1 = dh1^T x, db1 = column sums of dh1
    gemm(st, q->dh1b.as<bf16>(), 1, kHid, q->xb.as<bf16>(), kIn, 1, G + kW1, kIn, kHid, kIn, rows);
    k_colsum_part<<<dim3((unsigned)nparts, kHid / 256), 256, 0, st>>>(q->dh1.as<float>(), R, kHid, part);
    k_sum_parts<<<1, kHid, 0, st>>>(part, (int)nparts, kHid, G + kB1);
    QCP_CUDA(cudaGetLastError());
    if (grad_host) {
        QCP_CUDA(cudaMemcpyAsync(grad_host, G, 4 * kNParam, cudaMemcpyDeviceToHost, st));
    }
    // Adam
    q->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)q->step), c2 = 1.f - powf(b2, (float)q->step);
    k_adam<<<(unsigned)((kNParam + 255) / 256), 256, 0, st>>>(q->p.as<float>(), G, q->m.as<float>(), q->v.as<float>(),
                                                            kNParam, lr, b1, b2, 1e-8f, c1, c2, q->pb.as<bf16>());
    QCP_CUDA(cudaGetLastError());
    double loss = 0.0;
    QCP_CUDA(cudaMemcpyAsync(&loss, q->loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    QCP_CUDA(cudaStreamSynchronize(st));
    if (loss_host) *loss_host = loss;
    return QCP_OK;
}

int qcp_mlp_decode(const float* y, const float* offset, int64_t rows, double scale, double* warm_start,
                   double* precond_d, void* stream) {
    if (!y || rows < 0) {
        set_error("qcp_mlp_decode: null outputs or negative rows");
        return QCP_ERR_ARG;
    }
    if (rows == 0) return QCP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_decode<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(y, offset, rows, scale, warm_start, precond_d);
    QCP_CUDA(cudaGetLastError());
    QCP_CUDA(cudaStreamSynchronize(st));
    return QCP_OK;
}

int qcp_plan_features(qcp_plan* p, float* out) {
    if (!p || !out) {
        set_error("qcp_plan_features: null argument");
        return QCP_ERR_ARG;
    }
    if (p->kpsd || p->ndense) {
        set_error("qcp_plan_features: the features cover zero, R+ and SOC blocks; this plan has PSD, exp or power blocks");
        return QCP_ERR_ARG;
    }
    cudaStream_t st = p->stream;
    const int64_t Nt = p->N_tot;
    // host tables: row kind, M row, problem, SOC size and position
    std::vector<int8_t> kind(Nt), spos(Nt, 0);
    std::vector<int32_t> sdim(Nt, 0), pof(Nt);
    std::vector<int64_t> mrow(Nt);
    std::vector<double> kap(p->nprob);
    std::vector<Prob> dprob(p->nprob);  // kappa is computed on the device at plan time
    QCP_CUDA(cudaMemcpyAsync(dprob.data(), p->d_prob.p, sizeof(Prob) * p->nprob, cudaMemcpyDeviceToHost, st));
    QCP_CUDA(cudaStreamSynchronize(st));
    for (int pi = 0; pi < p->nprob; ++pi) {
        const Prob& pr = p->hprob[pi];
        kap[pi] = dprob[pi].kappa;
        const int64_t N = (int64_t)pr.n + pr.m + 1;
        for (int64_t r = 0; r < N; ++r) {
            kind[pr.doff + r] = r < pr.n ? 0 : (r == N - 1 ? 4 : 2);
            mrow[pr.doff + r] = pr.mrow + r;
            pof[pr.doff + r] = pi;
        }
        int64_t row = pr.n;
        for (size_t b = 0; b < p->cone_type[pi].size(); ++b) {
            const int t = p->cone_type[pi][b], d = p->cone_dim[pi][b];
            for (int k = 0; k < d; ++k) {
                const int64_t r = pr.doff + row + k;
                kind[r] = t == QCP_CONE_ZERO ? 1 : (t == QCP_CONE_NONNEG ? 2 : 3);
                if (t == QCP_CONE_SOC) {
                    sdim[r] = d;
                    spos[r] = k > 0;
                }
            }
            row += d;
        }
    }
    DevBuf dkind, dspos, dsdim, dpof, dmrow, dkap, dnorm, ddd;
    QCP_TRY(dkind.alloc(Nt));
    QCP_TRY(dspos.alloc(Nt));
    QCP_TRY(dsdim.alloc(4 * Nt));
    QCP_TRY(dpof.alloc(4 * Nt));
    QCP_TRY(dmrow.alloc(8 * Nt));
    QCP_TRY(dkap.alloc(8 * p->nprob));
    QCP_TRY(dnorm.alloc(8 * Nt));
    QCP_TRY(ddd.alloc(8 * Nt));
    QCP_CUDA(cudaMemcpyAsync(dkind.p, kind.data(), Nt, cudaMemcpyHostToDevice, st));
    QCP_CUDA(cudaMemcpyAsync(dspos.p, spos.data(), Nt, cudaMemcpyHostToDevice, st));
    QCP_CUDA(cudaMemcpyAsync(dsdim.p, sdim.data(), 4 * Nt, cudaMemcpyHostToDevice, st));
    QCP_CUDA(cudaMemcpyAsync(dpof.p, pof.data(), 4 * Nt, cudaMemcpyHostToDevice, st));
    QCP_CUDA(cudaMemcpyAsync(dmrow.p, mrow.data(), 8 * Nt, cudaMemcpyHostToDevice, st));
    QCP_CUDA(cudaMemcpyAsync(dkap.p, kap.data(), 8 * p->nprob, cudaMemcpyHostToDevice, st));
    const unsigned gb = (unsigned)((Nt + 255) / 256);
    if (p->dtype == QCP_F64)
        k_rownorm2<double><<<gb, 256, 0, st>>>(p->d_mrowptr.as<int64_t>(), p->d_mval.as<double>(),
                                               dmrow.as<int64_t>(), Nt, dnorm.as<double>());
    else
        k_rownorm2<float><<<gb, 256, 0, st>>>(p->d_mrowptr.as<int64_t>(), p->d_mval.as<float>(), dmrow.as<int64_t>(),
                                              Nt, dnorm.as<double>());
    // diagonal of D Pi: flags, then SOC blocks
    {
        std::vector<int8_t> hflag(Nt);
        QCP_CUDA(cudaMemcpyAsync(hflag.data(), p->d_flag.p, Nt, cudaMemcpyDeviceToHost, st));
        QCP_CUDA(cudaStreamSynchronize(st));
        std::vector<double> hd(Nt);
        for (int64_t r = 0; r < Nt; ++r) hd[r] = hflag[r] == RF_ONE ? 1.0 : 0.0;
        QCP_CUDA(cudaMemcpyAsync(ddd.p, hd.data(), 8 * Nt, cudaMemcpyHostToDevice, st));
        for (int pi = 0; pi < p->nprob; ++pi) {
            const Prob& pr = p->hprob[pi];
            if (pr.nsoc > 0)
                k_ddiag<<<(unsigned)((pr.nsoc + 255) / 256), 256, 0, st>>>(
                    p->d_flag.as<int8_t>() + pr.doff, p->d_blocks.as<SocBlock>() + pr.soff, pr.nsoc,
                    p->d_zy.as<double>() + pr.doff, ddd.as<double>() + pr.doff);
        }
        QCP_CUDA(cudaStreamSynchronize(st));
    }
    k_features<<<gb, 256, 0, st>>>(p->d_mrowptr.as<int64_t>(), dnorm.as<double>(), p->d_coefA.as<double>(),
                                   p->d_coefB.as<double>(), p->d_pz.as<double>(), p->d_zy.as<double>(),
                                   dkind.as<int8_t>(), ddd.as<double>(), dsdim.as<int32_t>(), dspos.as<int8_t>(), Nt,
                                   dmrow.as<int64_t>(), dkap.as<double>(), dpof.as<int32_t>(), out);
    QCP_CUDA(cudaGetLastError());
    QCP_CUDA(cudaStreamSynchronize(st));
    return QCP_OK;
}

int qcp_plan_scalings(const qcp_plan* p, double* rw, double* cd) {
    if (!p) {
        set_error("qcp_plan_scalings: null plan");
        return QCP_ERR_ARG;
    }
    if (rw) QCP_CUDA(cudaMemcpyAsync(rw, p->d_rw.p, 8 * (size_t)p->N_tot, cudaMemcpyDeviceToDevice, p->stream));
    if (cd) QCP_CUDA(cudaMemcpyAsync(cd, p->d_cd.p, 8 * (size_t)p->N_tot, cudaMemcpyDeviceToDevice, p->stream));
    QCP_CUDA(cudaStreamSynchronize(p->stream));
    return QCP_OK;
}

}  // extern "C"
