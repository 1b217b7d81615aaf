// Learned surrogate: a message-passing network on the SPH neighbour graph
// that predicts each particle's mean acceleration over the next k substeps.
//
// The paper has no learned part; the network is defined here (and in the
// header): node inputs x_a = [100 (rho_a/rho0 - 1), N_a (Eq. 20), C_a
// (Eq. 14), h |n_a| (Eq. 18)]; over the ordered pairs a != b with
// r_ab < 2h (Sec. 2-7) the edge weights, with V_b = m_b/rho_b and W, F of
// Eqs. 27-28,
//   w0 = V_b W_ab, w1 = V_b F_ab (x_a - x_b) h, w2 = V_b F_ab (y_a - y_b) h,
//   w3 = V_b F_ab ((u_a - u_b).(r_a - r_b)) h / U_ref;
// layers
//   h0 = relu(x W_in + b_in)
//   for l < 3:  z = h Pi_l;  g_a[32k + j] = sum_b w_k,ab z_b[j];
//               h = h + relu([h, g] U_l + c_l)
//   y = h D + d.
// Training runs in FP32 (SIMT GEMMs, the aggregation and its adjoint, Adam),
// as does the reference forward here; inference runs on the tensor cores
// (tcgen05, BF16 operands with FP32 accumulation) in sph_mpnn_tc.cu.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_mpnn.cuh"

using namespace sph;
using namespace mpnn;

namespace {

// ---------------------------------------------------------------------------
// node inputs, aggregation and its adjoint (one warp per particle)
// ---------------------------------------------------------------------------
__global__ void k_mp_inputs(PhysT<float> P, Hot<float> hot, Csf<float> csf, int n,
                            float *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4f h1 = hot.H1[i];
    V2f nh = csf.nhat[i];
    V2f nv = csf.nvec[i];
    x[4 * i + 0] = 100.0f * (h1.y / P.rho0 - 1.0f);
    x[4 * i + 1] = (nh.x != 0.0f || nh.y != 0.0f) ? 1.0f : 0.0f;
    x[4 * i + 2] = csf.C[i];
    x[4 * i + 3] = P.h * sqrtf(nv.x * nv.x + nv.y * nv.y);
}

// g_a[32k + lane] = sum_b w_k,ab z_b[lane]: the lanes evaluate 32 list entries
// at a time, then every valid pair is broadcast and accumulated.
template <int K>
__global__ void k_mp_aggregate(PhysT<float> P, Hot<float> hot, NList nl, int n, float inv_uref,
                               const float *__restrict__ z, float *__restrict__ g) {
    unsigned lane = threadIdx.x & 31u;
    unsigned a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= (unsigned)n) return;
    unsigned cnt = nl.cnt[a];
    const uint32_t *__restrict__ e = nl.e + (size_t)a * LIST_SLOTS;
    V4f ha = hot.H0[a];
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    for (unsigned base = 0; base < cnt; base += 32) {
        unsigned k = base + lane;
        unsigned o = 0;
        EdgeW ew{};
        bool ok = false;
        if (k < cnt) {
            float rx, ry, r2, du, dv;
            ok = list_pair(P, hot, e, k, a, ha, o, rx, ry, r2, du, dv);
            if (ok) ew = edge_weights<K>(P, rx, ry, r2, du, dv, hot.H1[o].x, inv_uref);
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1u;
            unsigned ob = __shfl_sync(0xffffffffu, o, src);
            float w0 = __shfl_sync(0xffffffffu, ew.w[0], src);
            float w1 = __shfl_sync(0xffffffffu, ew.w[1], src);
            float w2 = __shfl_sync(0xffffffffu, ew.w[2], src);
            float w3 = __shfl_sync(0xffffffffu, ew.w[3], src);
            float zb = z[(size_t)ob * MP_P + lane];
            acc0 += w0 * zb;
            acc1 += w1 * zb;
            acc2 += w2 * zb;
            acc3 += w3 * zb;
        }
    }
    float *ga = g + (size_t)a * MP_G;
    ga[0 * MP_P + lane] = acc0;
    ga[1 * MP_P + lane] = acc1;
    ga[2 * MP_P + lane] = acc2;
    ga[3 * MP_P + lane] = acc3;
}

// Adjoint: dz_b[lane] = sum over the pairs (a, b) of sum_k w_k,ab dg_a[32k +
// lane], gathered over b's own list (the pair relation is symmetric).  Seen
// from b, the pair's offsets are r_b - r_a = -(r_a - r_b), so w1 and w2
// change sign while w0 and w3 do not, and the volume is b's own.
template <int K>
__global__ void k_mp_aggregate_T(PhysT<float> P, Hot<float> hot, NList nl, int n, float inv_uref,
                                 const float *__restrict__ dg, float *__restrict__ dz) {
    unsigned lane = threadIdx.x & 31u;
    unsigned b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= (unsigned)n) return;
    unsigned cnt = nl.cnt[b];
    const uint32_t *__restrict__ e = nl.e + (size_t)b * LIST_SLOTS;
    V4f hb = hot.H0[b];
    float Vb = hot.H1[b].x;
    float acc = 0.f;
    for (unsigned base = 0; base < cnt; base += 32) {
        unsigned k = base + lane;
        unsigned o = 0;
        EdgeW ew{};
        bool ok = false;
        if (k < cnt) {
            float rx, ry, r2, du, dv;
            ok = list_pair(P, hot, e, k, b, hb, o, rx, ry, r2, du, dv);
            // weights of the pair (o, b): r_o - r_b = -(rx, ry), u_o - u_b = -(du, dv)
            if (ok) ew = edge_weights<K>(P, -rx, -ry, r2, -du, -dv, Vb, inv_uref);
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1u;
            unsigned oa = __shfl_sync(0xffffffffu, o, src);
            float w0 = __shfl_sync(0xffffffffu, ew.w[0], src);
            float w1 = __shfl_sync(0xffffffffu, ew.w[1], src);
            float w2 = __shfl_sync(0xffffffffu, ew.w[2], src);
            float w3 = __shfl_sync(0xffffffffu, ew.w[3], src);
            const float *da = dg + (size_t)oa * MP_G;
            acc += w0 * da[lane] + w1 * da[MP_P + lane] + w2 * da[2 * MP_P + lane] +
                   w3 * da[3 * MP_P + lane];
        }
    }
    dz[(size_t)b * MP_P + lane] = acc;
}

// Edge list for inspection: one warp per particle writes its valid pairs at
// slots reserved with one atomic per warp.
template <int K>
__global__ void k_mp_edges(PhysT<float> P, Hot<float> hot, NList nl, int n, float inv_uref,
                           unsigned long long *__restrict__ count, long long cap,
                           int *__restrict__ ea, int *__restrict__ eb, float *__restrict__ w) {
    unsigned lane = threadIdx.x & 31u;
    unsigned a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= (unsigned)n) return;
    unsigned cnt = nl.cnt[a];
    const uint32_t *__restrict__ e = nl.e + (size_t)a * LIST_SLOTS;
    V4f ha = hot.H0[a];
    for (unsigned base = 0; base < cnt; base += 32) {
        unsigned k = base + lane;
        unsigned o = 0;
        EdgeW ew{};
        bool ok = false;
        if (k < cnt) {
            float rx, ry, r2, du, dv;
            ok = list_pair(P, hot, e, k, a, ha, o, rx, ry, r2, du, dv);
            if (ok) ew = edge_weights<K>(P, rx, ry, r2, du, dv, hot.H1[o].x, inv_uref);
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        unsigned long long slot0 = 0;
        if (lane == 0 && m) slot0 = atomicAdd(count, (unsigned long long)__popc(m));
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        if (ok) {
            unsigned long long slot = slot0 + __popc(m & ((1u << lane) - 1u));
            if ((long long)slot < cap) {
                ea[slot] = (int)a;
                eb[slot] = (int)o;
                for (int c = 0; c < 4; ++c) w[4 * slot + c] = ew.w[c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 SIMT GEMMs (training path, and the thin layers of inference)
// ---------------------------------------------------------------------------
enum Epi { EPI_STORE = 0, EPI_RELU = 1, EPI_RESRELU = 2, EPI_ACCUM = 3 };

constexpr int GM_ROWS = 64, GM_KC = 32;

// C[M x N] = A[M x K] * B (+ bias) with an epilogue; A(m, k) is A0[m*lda0 + k]
// for k < K0 and A1[m*lda1 + k - K0] above (a column concatenation); B(k, n)
// is B[k*ldb + n], or B[n*ldb + k] when transB.  N <= 128.  Block: 32 x 8
// threads, 64 rows; thread (tx, ty) owns rows ty*8 .. ty*8+7, columns
// 4tx .. 4tx+3.  EPI_RELU/EPI_RESRELU also store the pre-activation to Pre
// (if given); EPI_RESRELU adds relu(.) to R.
template <int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float *__restrict__ A0,
                                              int lda0, int K0, const float *__restrict__ A1,
                                              int lda1, const float *__restrict__ B, int ldb,
                                              int transB, const float *__restrict__ bias,
                                              const float *R, float *Pre, float *C, int ldc) {
    __shared__ float As[GM_KC][GM_ROWS + 1];
    __shared__ __align__(16) float Bs[GM_KC][128];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int m0 = blockIdx.x * GM_ROWS;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int k0 = 0; k0 < K; k0 += GM_KC) {
        for (int t = tid; t < GM_ROWS * GM_KC; t += 256) {
            int r = t / GM_KC, kk = t % GM_KC;
            int m = m0 + r, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < K) v = k < K0 ? A0[(size_t)m * lda0 + k] : A1[(size_t)m * lda1 + (k - K0)];
            As[kk][r] = v;
        }
        for (int t = tid; t < GM_KC * 128; t += 256) {
            int kk = t / 128, nn = t % 128;
            int k = k0 + kk;
            float v = 0.f;
            if (k < K && nn < N) v = transB ? B[(size_t)nn * ldb + k] : B[(size_t)k * ldb + nn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GM_KC; ++kk) {
            float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tx]);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                float a = As[kk][ty * 8 + r];
                acc[r][0] += a * b.x;
                acc[r][1] += a * b.y;
                acc[r][2] += a * b.z;
                acc[r][3] += a * b.w;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int m = m0 + ty * 8 + r;
        if (m >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int nn = 4 * tx + c;
            if (nn >= N) continue;
            float v = acc[r][c] + (bias ? bias[nn] : 0.f);
            size_t at = (size_t)m * ldc + nn;
            if (EPI == EPI_STORE) {
                C[at] = v;
            } else if (EPI == EPI_RELU) {
                if (Pre) Pre[at] = v;
                C[at] = v > 0.f ? v : 0.f;
            } else if (EPI == EPI_RESRELU) {
                if (Pre) Pre[at] = v;
                C[at] = R[at] + (v > 0.f ? v : 0.f);
            } else {
                C[at] += acc[r][c];
            }
        }
    }
}

constexpr int GT_ROWS = 256;   // rows of M per block of the weight-gradient GEMM

// dB[K x N] += A^T dC over a chunk of rows (A as in k_gemm), and dbias[N] +=
// column sums of dC (blocks with blockIdx.x == 0).  Block: 32 x 8 threads, a
// 32 (k) x 32 (n) tile; thread (tx, ty) owns k = ty*4 .. ty*4+3, n = tx.
__global__ void __launch_bounds__(256) k_gemm_tn(int M, int N, int K, const float *__restrict__ A0,
                                                 int lda0, int K0, const float *__restrict__ A1,
                                                 int lda1, const float *__restrict__ dC, int ldc,
                                                 float *dB, float *dbias) {
    __shared__ float As[32][33];
    __shared__ float Cs[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int k0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
    const int mbeg = blockIdx.z * GT_ROWS, mend = min(M, mbeg + GT_ROWS);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float bsum = 0.f;
    for (int m0 = mbeg; m0 < mend; m0 += 32) {
        for (int t = tid; t < 32 * 32; t += 256) {
            int r = t / 32, c = t % 32;
            int m = m0 + r, k = k0 + c, nn = n0 + c;
            float va = 0.f, vc = 0.f;
            if (m < mend && k < K) va = k < K0 ? A0[(size_t)m * lda0 + k] : A1[(size_t)m * lda1 + (k - K0)];
            if (m < mend && nn < N) vc = dC[(size_t)m * ldc + nn];
            As[r][c] = va;
            Cs[r][c] = vc;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            float c = Cs[r][tx];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] += As[r][ty * 4 + j] * c;
            if (ty == 0) bsum += c;
        }
        __syncthreads();
    }
    int nn = n0 + tx;
    if (nn >= N) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int k = k0 + ty * 4 + j;
        if (k < K) atomicAdd(&dB[(size_t)k * N + nn], acc[j]);
    }
    if (dbias && blockIdx.x == 0 && ty == 0) atomicAdd(&dbias[nn], bsum);
}

// ---------------------------------------------------------------------------
// loss and optimiser
// ---------------------------------------------------------------------------
// L = (1/n) sum |y - t|^2; dy = 2 (y - t) / n.
__global__ void k_mp_loss(int n, const float *__restrict__ y, const float *__restrict__ t,
                          float *__restrict__ dy, double *loss) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        float d0 = y[2 * i] - t[2 * i], d1 = y[2 * i + 1] - t[2 * i + 1];
        dy[2 * i] = 2.f * d0 / (float)n;
        dy[2 * i + 1] = 2.f * d1 / (float)n;
        s = ((double)d0 * d0 + (double)d1 * d1) / (double)n;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b += ws[k];
        atomicAdd(loss, b);
    }
}

// Adam (bias-corrected step sizes passed in: a1 = lr / (1 - b1^t), a2 =
// 1 / (1 - b2^t)).
__global__ void k_adam(long long np, float *__restrict__ p, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float b1, float b2,
                       float a1, float a2, float eps) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= a1 * mi / (sqrtf(vi * a2) + eps);
}

__global__ void k_relu_mask(long long nel, const float *__restrict__ pre, float *__restrict__ d) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nel && !(pre[i] > 0.f)) d[i] = 0.f;
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// the network object
// ---------------------------------------------------------------------------
struct sph_mpnn {
    int device = 0;
    long long cap = 0;
    std::string err;
    cudaStream_t stream = nullptr;   // the context's stream of the last call
    std::vector<void *> allocs;
    float *param = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    long long adam_t = 0;
    // BF16 weight images of the tensor-core pass (rebuilt after a parameter
    // change) and its scratch for sph_mpnn_forward
    __nv_bfloat16 *u_img = nullptr, *pi_img = nullptr;
    bool img_stale = true;
    MpScratchHandle *fast = nullptr;
    int stall = 0;                   // sph_mpnn_inject_stall
    // activations (capacity rows)
    float *x = nullptr, *pre_in = nullptr, *h[MP_L + 1] = {}, *z[MP_L] = {}, *g[MP_L] = {},
          *pre[MP_L] = {}, *y = nullptr;
    // backward scratch
    float *t = nullptr, *dy = nullptr, *dh = nullptr, *dcat = nullptr /* dpre */, *dz = nullptr,
          *dtmp = nullptr /* dg */;
    double *loss = nullptr;
    unsigned long long *ecount = nullptr;
};

namespace {

std::string g_mp_error;

sph_status mp_fail(sph_mpnn *n, sph_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (n) n->err = buf; else g_mp_error = buf;
    return st;
}

#define MCK(net, call, what)                                                                      \
    do {                                                                                          \
        cudaError_t ce_ = (call);                                                                 \
        if (ce_ != cudaSuccess)                                                                   \
            return mp_fail((net), ce_ == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA,  \
                           "%s: %s", (what), cudaGetErrorString(ce_));                            \
    } while (0)

template <class T> sph_status mp_alloc(sph_mpnn *n, T **p, size_t count) {
    void *q = nullptr;
    MCK(n, cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)), "allocation");
    n->allocs.push_back(q);
    *p = (T *)q;
    return SPH_OK;
}

// A view of an evaluated FP32 context, checked.
sph_status mp_view(sph_mpnn *net, sph_ctx *ctx, CtxView &v) {
    if (!ctx) return mp_fail(net, SPH_ERR_ARG, "context is NULL");
    ctx_view(ctx, &v);
    if (!v.fp32) return mp_fail(net, SPH_ERR_ARG, "the surrogate needs an FP32 context");
    if (!v.evaluated) return mp_fail(net, SPH_ERR_STATE, "call sph_evaluate on the context first");
    if (v.device != net->device) return mp_fail(net, SPH_ERR_ARG, "context on another device");
    if (v.n > net->cap) return mp_fail(net, SPH_ERR_CAPACITY, "%d particles exceed capacity %lld", v.n, net->cap);
    net->stream = v.stream;
    return SPH_OK;
}

void gemm(cudaStream_t s, int epi, int M, int N, int K, const float *A0, int lda0, int K0,
          const float *A1, int lda1, const float *B, int ldb, int transB, const float *bias,
          const float *R, float *Pre, float *C, int ldc) {
    if (M <= 0) return;
    dim3 grid(nblk(M, GM_ROWS)), block(32, 8);
    switch (epi) {
    case EPI_STORE:
        k_gemm<EPI_STORE><<<grid, block, 0, s>>>(M, N, K, A0, lda0, K0, A1, lda1, B, ldb, transB, bias, R, Pre, C, ldc);
        break;
    case EPI_RELU:
        k_gemm<EPI_RELU><<<grid, block, 0, s>>>(M, N, K, A0, lda0, K0, A1, lda1, B, ldb, transB, bias, R, Pre, C, ldc);
        break;
    case EPI_RESRELU:
        k_gemm<EPI_RESRELU><<<grid, block, 0, s>>>(M, N, K, A0, lda0, K0, A1, lda1, B, ldb, transB, bias, R, Pre, C, ldc);
        break;
    default:
        k_gemm<EPI_ACCUM><<<grid, block, 0, s>>>(M, N, K, A0, lda0, K0, A1, lda1, B, ldb, transB, bias, R, Pre, C, ldc);
    }
}

void gemm_tn(cudaStream_t s, int M, int N, int K, const float *A0, int lda0, int K0,
             const float *A1, int lda1, const float *dC, int ldc, float *dB, float *dbias) {
    if (M <= 0) return;
    dim3 grid(nblk(K, 32), nblk(N, 32), nblk(M, GT_ROWS)), block(32, 8);
    k_gemm_tn<<<grid, block, 0, s>>>(M, N, K, A0, lda0, K0, A1, lda1, dC, ldc, dB, dbias);
}

template <class F> void with_kernel(int kernel, F &&f) {
    if (kernel == 1) f(std::integral_constant<int, 1>{});
    else f(std::integral_constant<int, 0>{});
}

// FP32 forward pass over the n particles of the view, keeping every
// activation for the backward pass (training; the reference for the
// tensor-core pass of sph_mpnn_tc.cu).
sph_status mp_forward(sph_mpnn *net, const CtxView &v, float inv_uref) {
    cudaStream_t s = v.stream;
    const int n = v.n;
    const Layout &L = kMP;
    const float *P = net->param;
    if (n == 0) return SPH_OK;
    k_mp_inputs<<<nblk(n, 256), 256, 0, s>>>(v.P, v.hot, v.csf, n, net->x);
    gemm(s, EPI_RELU, n, MP_H, MP_IN, net->x, MP_IN, MP_IN, nullptr, 0, P + L.W_in, MP_H, 0,
         P + L.b_in, nullptr, net->pre_in, net->h[0], MP_H);
    for (int l = 0; l < MP_L; ++l) {
        gemm(s, EPI_STORE, n, MP_P, MP_H, net->h[l], MP_H, MP_H, nullptr, 0, P + L.Pi[l], MP_P, 0,
             nullptr, nullptr, nullptr, net->z[l], MP_P);
        with_kernel(v.P.kernel, [&](auto Kc) {
            constexpr int K = decltype(Kc)::value;
            k_mp_aggregate<K><<<nblk((long long)n * 32, 256), 256, 0, s>>>(
                v.P, v.hot, v.nl, n, inv_uref, net->z[l], net->g[l]);
        });
        gemm(s, EPI_RESRELU, n, MP_H, MP_CAT, net->h[l], MP_H, MP_H, net->g[l], MP_G, P + L.U[l],
             MP_H, 0, P + L.c[l], net->h[l], net->pre[l], net->h[l + 1], MP_H);
    }
    gemm(s, EPI_STORE, n, MP_OUT, MP_H, net->h[MP_L], MP_H, MP_H, nullptr, 0, P + L.D, MP_OUT, 0,
         P + L.d, nullptr, nullptr, net->y, MP_OUT);
    MCK(net, cudaGetLastError(), "forward launch");
    return SPH_OK;
}

// Backward pass of the FP32 forward; fills net->grad (overwritten).
sph_status mp_backward(sph_mpnn *net, const CtxView &v, float inv_uref) {
    cudaStream_t s = v.stream;
    const int n = v.n;
    const Layout &L = kMP;
    const float *P = net->param;
    float *G = net->grad;
    MCK(net, cudaMemsetAsync(G, 0, (size_t)L.total * sizeof(float), s), "clear gradients");
    if (n == 0) return SPH_OK;
    // output layer
    gemm_tn(s, n, MP_OUT, MP_H, net->h[MP_L], MP_H, MP_H, nullptr, 0, net->dy, MP_OUT, G + L.D, G + L.d);
    gemm(s, EPI_STORE, n, MP_H, MP_OUT, net->dy, MP_OUT, MP_OUT, nullptr, 0, P + L.D, MP_OUT, 1,
         nullptr, nullptr, nullptr, net->dh, MP_H);
    const long long nh = (long long)n * MP_H;
    float *dpre = net->dcat, *dg = net->dtmp;
    for (int l = MP_L - 1; l >= 0; --l) {
        // dpre = dh * (pre > 0)
        MCK(net, cudaMemcpyAsync(dpre, net->dh, nh * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy");
        k_relu_mask<<<nblk(nh, 256), 256, 0, s>>>(nh, net->pre[l], dpre);
        gemm_tn(s, n, MP_H, MP_CAT, net->h[l], MP_H, MP_H, net->g[l], MP_G, dpre, MP_H,
                G + L.U[l], G + L.c[l]);
        // [dh_h, dg] = dpre U^T, split by the rows of U: dh += dpre U[:H]^T,
        // dg = dpre U[H:]^T
        gemm(s, EPI_ACCUM, n, MP_H, MP_H, dpre, MP_H, MP_H, nullptr, 0, P + L.U[l], MP_H, 1,
             nullptr, nullptr, nullptr, net->dh, MP_H);
        gemm(s, EPI_STORE, n, MP_G, MP_H, dpre, MP_H, MP_H, nullptr, 0, P + L.U[l] + MP_H * MP_H,
             MP_H, 1, nullptr, nullptr, nullptr, dg, MP_G);
        with_kernel(v.P.kernel, [&](auto Kc) {
            constexpr int K = decltype(Kc)::value;
            k_mp_aggregate_T<K><<<nblk((long long)n * 32, 256), 256, 0, s>>>(
                v.P, v.hot, v.nl, n, inv_uref, dg, net->dz);
        });
        gemm_tn(s, n, MP_P, MP_H, net->h[l], MP_H, MP_H, nullptr, 0, net->dz, MP_P, G + L.Pi[l], nullptr);
        // dh += dz Pi^T
        gemm(s, EPI_ACCUM, n, MP_H, MP_P, net->dz, MP_P, MP_P, nullptr, 0, P + L.Pi[l], MP_P, 1,
             nullptr, nullptr, nullptr, net->dh, MP_H);
    }
    k_relu_mask<<<nblk(nh, 256), 256, 0, s>>>(nh, net->pre_in, net->dh);
    gemm_tn(s, n, MP_H, MP_IN, net->x, MP_IN, MP_IN, nullptr, 0, net->dh, MP_H, G + L.W_in, G + L.b_in);
    MCK(net, cudaGetLastError(), "backward launch");
    return SPH_OK;
}

}  // namespace

// Scratch of the tensor-core pass, owned by a context or by the network.
struct MpScratchHandle {
    MpScratch s;
    int device = -1;
    std::vector<void *> allocs;
};

void mpnn_scratch_free(MpScratchHandle *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    for (void *p : h->allocs) cudaFree(p);
    delete h;
}

namespace {

// *hp holds room for cap particles on the device afterwards.
sph_status scratch_ensure(sph_mpnn *net, MpScratchHandle **hp, long long cap, int device) {
    if (*hp && (*hp)->s.cap >= cap && (*hp)->device == device) return SPH_OK;
    mpnn_scratch_free(*hp);
    *hp = nullptr;
    MpScratchHandle *h = new (std::nothrow) MpScratchHandle();
    if (!h) return mp_fail(net, SPH_ERR_OOM, "host allocation failed");
    h->device = device;
    const size_t C = (size_t)std::max<long long>(cap, 1);
    const size_t bytes[6] = {C * LIST_SLOTS * sizeof(uint4), C * sizeof(unsigned), C * MP_H * 2,
                             C * MP_P * 2, C * MP_P * 2, C * sizeof(float2)};
    void *p[6] = {};
    for (int k = 0; k < 6; ++k) {
        cudaError_t e = cudaMalloc(&p[k], bytes[k]);
        if (e != cudaSuccess) {
            mpnn_scratch_free(h);
            return mp_fail(net, e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA,
                           "inference scratch: %s", cudaGetErrorString(e));
        }
        h->allocs.push_back(p[k]);
    }
    h->s.edge = (uint4 *)p[0];
    h->s.ecnt = (unsigned *)p[1];
    h->s.h = (__nv_bfloat16 *)p[2];
    h->s.z[0] = (__nv_bfloat16 *)p[3];
    h->s.z[1] = (__nv_bfloat16 *)p[4];
    h->s.y = (float2 *)p[5];
    h->s.cap = (long long)C;
    *hp = h;
    return SPH_OK;
}

// The tensor-core inference pass of the view into scratch h (sph_mpnn_tc.cu).
sph_status mp_fast(sph_mpnn *net, const CtxView &v, float inv_uref, MpScratchHandle *h) {
    if (net->img_stale) {
        tc_weight_images(net->param, net->u_img, net->pi_img, v.stream);
        MCK(net, cudaStreamSynchronize(v.stream), "weight images");
        net->img_stale = false;
    }
    MCK(net, tc_forward(v, inv_uref, net->param, net->u_img, net->pi_img, h->s, v.err,
                        net->stall),
        "tensor-core forward");
    return SPH_OK;
}

}  // namespace

sph_status mpnn_predict(sph_mpnn *net, sph_ctx *c, double u_ref, bool bf16, const float2 **y,
                        MpScratchHandle **scratch) {
    if (!net || !y || !scratch || !(u_ref > 0))
        return net ? mp_fail(net, SPH_ERR_ARG, "bad arguments") : SPH_ERR_ARG;
    CtxView v;
    sph_status s = mp_view(net, c, v);
    if (s) return s;
    if (!bf16) {
        s = mp_forward(net, v, (float)(1.0 / u_ref));
        *y = reinterpret_cast<const float2 *>(net->y);
        return s;
    }
    s = scratch_ensure(net, scratch, v.cap, v.device);
    if (s) return s;
    s = mp_fast(net, v, (float)(1.0 / u_ref), *scratch);
    *y = (*scratch)->s.y;
    return s;
}

extern "C" {

long long sph_mpnn_param_count(void) { return kMP.total; }

const char *sph_mpnn_last_error(const sph_mpnn *net) {
    return net ? net->err.c_str() : g_mp_error.c_str();
}

void sph_mpnn_destroy(sph_mpnn *net) {
    if (!net) return;
    cudaSetDevice(net->device);
    cudaDeviceSynchronize();
    mpnn_scratch_free(net->fast);
    for (void *p : net->allocs) cudaFree(p);
    delete net;
}

sph_status sph_mpnn_create(int device, long long capacity, sph_mpnn **out) {
    if (!out) return mp_fail(nullptr, SPH_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (capacity < 1 || capacity > (1ll << 26))
        return mp_fail(nullptr, SPH_ERR_ARG, "capacity must lie in [1, 2^26]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return mp_fail(nullptr, SPH_ERR_ARG, "device %d not available", device);
    sph_mpnn *net = new (std::nothrow) sph_mpnn();
    if (!net) return mp_fail(nullptr, SPH_ERR_OOM, "host allocation failed");
    net->device = device;
    net->cap = capacity;
    auto bail = [&](sph_status st) {
        g_mp_error = net->err;
        sph_mpnn_destroy(net);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(mp_fail(net, SPH_ERR_CUDA, "cudaSetDevice"));
    const size_t C = (size_t)capacity, NP = (size_t)kMP.total;
    sph_status s = SPH_OK;
    auto A = [&](float **p, size_t cnt) { if (!s) s = mp_alloc(net, p, cnt); };
    A(&net->param, NP); A(&net->grad, NP); A(&net->am, NP); A(&net->av, NP);
    A(&net->x, C * MP_IN); A(&net->pre_in, C * MP_H);
    for (int l = 0; l <= MP_L; ++l) A(&net->h[l], C * MP_H);
    for (int l = 0; l < MP_L; ++l) { A(&net->z[l], C * MP_P); A(&net->g[l], C * MP_G); A(&net->pre[l], C * MP_H); }
    A(&net->y, C * MP_OUT); A(&net->t, C * MP_OUT); A(&net->dy, C * MP_OUT);
    A(&net->dh, C * MP_H); A(&net->dcat, C * MP_H); A(&net->dz, C * MP_P); A(&net->dtmp, C * MP_G);
    if (!s) s = mp_alloc(net, &net->u_img, MP_L * TC_U_BYTES / 2);
    if (!s) s = mp_alloc(net, &net->pi_img, MP_L * TC_PI_BYTES / 2);
    if (!s) s = mp_alloc(net, &net->loss, 1);
    if (!s) s = mp_alloc(net, &net->ecount, 1);
    if (s) return bail(s);
    if (cudaMemset(net->param, 0, NP * 4) != cudaSuccess || cudaMemset(net->am, 0, NP * 4) != cudaSuccess ||
        cudaMemset(net->av, 0, NP * 4) != cudaSuccess || cudaMemset(net->grad, 0, NP * 4) != cudaSuccess)
        return bail(mp_fail(net, SPH_ERR_CUDA, "clear"));
    *out = net;
    return SPH_OK;
}

sph_status sph_mpnn_set_params(sph_mpnn *net, const float *host, long long n) {
    if (!net || !host || n != kMP.total) return net ? mp_fail(net, SPH_ERR_ARG, "expected %lld parameters", kMP.total) : SPH_ERR_ARG;
    MCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    MCK(net, cudaMemcpy(net->param, host, (size_t)n * 4, cudaMemcpyHostToDevice), "upload parameters");
    MCK(net, cudaMemset(net->am, 0, (size_t)n * 4), "reset optimiser");
    MCK(net, cudaMemset(net->av, 0, (size_t)n * 4), "reset optimiser");
    net->adam_t = 0;
    net->img_stale = true;
    return SPH_OK;
}

sph_status sph_mpnn_get_params(sph_mpnn *net, float *host, long long n) {
    if (!net || !host || n != kMP.total) return net ? mp_fail(net, SPH_ERR_ARG, "expected %lld parameters", kMP.total) : SPH_ERR_ARG;
    MCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    MCK(net, cudaDeviceSynchronize(), "synchronize");
    MCK(net, cudaMemcpy(host, net->param, (size_t)n * 4, cudaMemcpyDeviceToHost), "download parameters");
    return SPH_OK;
}

sph_status sph_mpnn_get_grads(sph_mpnn *net, float *host, long long n) {
    if (!net || !host || n != kMP.total) return net ? mp_fail(net, SPH_ERR_ARG, "expected %lld parameters", kMP.total) : SPH_ERR_ARG;
    MCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    MCK(net, cudaDeviceSynchronize(), "synchronize");
    MCK(net, cudaMemcpy(host, net->grad, (size_t)n * 4, cudaMemcpyDeviceToHost), "download gradients");
    return SPH_OK;
}

sph_status sph_mpnn_features(sph_mpnn *net, sph_ctx *ctx, double u_ref, long long cap, long long *n,
                             unsigned *id, float *x, long long ecap, long long *ne, int *ea, int *eb,
                             float *w) {
    if (!net || !n || !ne || !(u_ref > 0)) return net ? mp_fail(net, SPH_ERR_ARG, "bad arguments") : SPH_ERR_ARG;
    CtxView v;
    sph_status s = mp_view(net, ctx, v);
    if (s) return s;
    *n = v.n;
    if (v.n > cap || (v.n > 0 && (!id || !x))) return mp_fail(net, SPH_ERR_CAPACITY, "need room for %d particles", v.n);
    cudaStream_t st = v.stream;
    float inv = (float)(1.0 / u_ref);
    MCK(net, cudaMemsetAsync(net->ecount, 0, sizeof(unsigned long long), st), "clear");
    if (v.n > 0) {
        k_mp_inputs<<<nblk(v.n, 256), 256, 0, st>>>(v.P, v.hot, v.csf, v.n, net->x);
        // edges go straight to pinned/host-visible memory only through a
        // device staging copy: use the activation buffers as scratch
        with_kernel(v.P.kernel, [&](auto Kc) {
            constexpr int K = decltype(Kc)::value;
            k_mp_edges<K><<<nblk((long long)v.n * 32, 256), 256, 0, st>>>(
                v.P, v.hot, v.nl, v.n, inv, net->ecount, 0, nullptr, nullptr, nullptr);
        });
    }
    unsigned long long ecount = 0;
    MCK(net, cudaMemcpyAsync(&ecount, net->ecount, 8, cudaMemcpyDeviceToHost, st), "count");
    MCK(net, cudaStreamSynchronize(st), "synchronize");
    *ne = (long long)ecount;
    if ((long long)ecount > ecap || (ecount > 0 && (!ea || !eb || !w)))
        return mp_fail(net, SPH_ERR_CAPACITY, "need room for %llu edges", ecount);
    std::vector<int> hea(ecount), heb(ecount);
    std::vector<float> hw(4 * ecount);
    if (ecount > 0) {
        int *dea = nullptr, *deb = nullptr;
        float *dw = nullptr;
        MCK(net, cudaMalloc(&dea, ecount * 4), "edge scratch");
        cudaMalloc(&deb, ecount * 4);
        cudaMalloc(&dw, ecount * 16);
        cudaMemsetAsync(net->ecount, 0, sizeof(unsigned long long), st);
        with_kernel(v.P.kernel, [&](auto Kc) {
            constexpr int K = decltype(Kc)::value;
            k_mp_edges<K><<<nblk((long long)v.n * 32, 256), 256, 0, st>>>(
                v.P, v.hot, v.nl, v.n, inv, net->ecount, (long long)ecount, dea, deb, dw);
        });
        cudaMemcpyAsync(ea, dea, ecount * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(eb, deb, ecount * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(w, dw, ecount * 16, cudaMemcpyDeviceToHost, st);
        cudaError_t ce = cudaStreamSynchronize(st);
        cudaFree(dea);
        cudaFree(deb);
        cudaFree(dw);
        MCK(net, ce, "edges");
    }
    if (v.n > 0) {
        MCK(net, cudaMemcpyAsync(x, net->x, (size_t)v.n * 16, cudaMemcpyDeviceToHost, st), "inputs");
        MCK(net, cudaMemcpyAsync(id, v.id, (size_t)v.n * 4, cudaMemcpyDeviceToHost, st), "ids");
        MCK(net, cudaStreamSynchronize(st), "synchronize");
    }
    return SPH_OK;
}

sph_status sph_mpnn_forward(sph_mpnn *net, sph_ctx *ctx, double u_ref, int bf16, long long cap,
                            long long *n, unsigned *id, float *y) {
    if (!net || !n || !(u_ref > 0)) return net ? mp_fail(net, SPH_ERR_ARG, "bad arguments") : SPH_ERR_ARG;
    CtxView v;
    sph_status s = mp_view(net, ctx, v);
    if (s) return s;
    *n = v.n;
    if (v.n > cap || (v.n > 0 && (!id || !y))) return mp_fail(net, SPH_ERR_CAPACITY, "need room for %d particles", v.n);
    const float *dev_y = net->y;
    if (bf16) {
        s = scratch_ensure(net, &net->fast, net->cap, net->device);
        if (!s) s = mp_fast(net, v, (float)(1.0 / u_ref), net->fast);
        if (!s) dev_y = reinterpret_cast<const float *>(net->fast->s.y);
    } else {
        s = mp_forward(net, v, (float)(1.0 / u_ref));
    }
    if (s) return s;
    if (v.n > 0) {
        MCK(net, cudaMemcpyAsync(y, dev_y, (size_t)v.n * 8, cudaMemcpyDeviceToHost, v.stream), "outputs");
        MCK(net, cudaMemcpyAsync(id, v.id, (size_t)v.n * 4, cudaMemcpyDeviceToHost, v.stream), "ids");
    }
    unsigned err = 0;
    if (bf16) MCK(net, cudaMemcpyAsync(&err, v.err, sizeof err, cudaMemcpyDeviceToHost, v.stream), "error word");
    MCK(net, cudaStreamSynchronize(v.stream), "synchronize");
    if (err & ERR_TIMEOUT)
        return mp_fail(net, SPH_ERR_TIMEOUT, "a bounded wait of the inference pass ran out");
    return SPH_OK;
}

sph_status sph_mpnn_backward(sph_mpnn *net, sph_ctx *ctx, double u_ref, const float *target,
                             long long n, double *loss) {
    if (!net || !(u_ref > 0)) return net ? mp_fail(net, SPH_ERR_ARG, "bad arguments") : SPH_ERR_ARG;
    CtxView v;
    sph_status s = mp_view(net, ctx, v);
    if (s) return s;
    if (n != v.n || (n > 0 && !target)) return mp_fail(net, SPH_ERR_ARG, "target must hold %d rows", v.n);
    float inv = (float)(1.0 / u_ref);
    s = mp_forward(net, v, inv);
    if (s) return s;
    cudaStream_t st = v.stream;
    MCK(net, cudaMemsetAsync(net->loss, 0, sizeof(double), st), "clear loss");
    if (n > 0) {
        MCK(net, cudaMemcpyAsync(net->t, target, (size_t)n * 8, cudaMemcpyHostToDevice, st), "target");
        k_mp_loss<<<nblk(n, 256), 256, 0, st>>>((int)n, net->y, net->t, net->dy, net->loss);
    }
    s = mp_backward(net, v, inv);
    if (s) return s;
    double l = 0.0;
    MCK(net, cudaMemcpyAsync(&l, net->loss, sizeof(double), cudaMemcpyDeviceToHost, st), "loss");
    MCK(net, cudaStreamSynchronize(st), "synchronize");
    if (loss) *loss = l;
    if (!std::isfinite(l)) return mp_fail(net, SPH_ERR_NONFINITE, "non-finite loss");
    return SPH_OK;
}

sph_status sph_mpnn_inject_stall(sph_mpnn *net, int on) {
    if (!net) return SPH_ERR_ARG;
    net->stall = on != 0;
    return SPH_OK;
}

sph_status sph_mpnn_adam(sph_mpnn *net, double lr) {
    if (!net || !(lr > 0)) return net ? mp_fail(net, SPH_ERR_ARG, "lr must be > 0") : SPH_ERR_ARG;
    const float b1 = 0.9f, b2 = 0.999f;
    net->adam_t += 1;
    float a1 = (float)(lr / (1.0 - std::pow((double)b1, (double)net->adam_t)));
    float a2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)net->adam_t)));
    MCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    k_adam<<<nblk(kMP.total, 256), 256, 0, net->stream>>>(kMP.total, net->param, net->grad, net->am,
                                                          net->av, b1, b2, a1, a2, 1e-8f);
    net->img_stale = true;
    MCK(net, cudaGetLastError(), "adam");
    return SPH_OK;
}

}  // extern "C"
