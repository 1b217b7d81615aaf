// Tensor-core inference pass of the learned surrogate (the network of
// sph_mpnn.cu: node inputs, three message-passing layers, output layer).
//
// One persistent kernel per layer, one CTA of 25 warps per SM, over tiles of
// TC_M = 128 particles in cell order:
//   * the layer's weights (U_l^T, Pi_{l+1}^T as BF16 core-matrix images) are
//     copied once per CTA into shared memory with cp.async.bulk;
//   * per tile, the hidden state h_l arrives by TMA (cp.async.bulk.tensor,
//     16 boxes of 128 rows x 8 columns) while 16 warps aggregate the
//     messages g_a[32k + j] = sum_b w_k,ab z_b[j] from precomputed edge
//     records, four threads per particle, straight into the operand tile;
//   * one thread issues tcgen05.mma (kind::f16, BF16 operands, FP32
//     accumulators in tensor memory) for [h, g] U_l^T, 8 epilogue warps read
//     the accumulators back with tcgen05.ld and form h_{l+1} = h_l + relu(. +
//     c_l), which goes to global memory and, in place, back into the operand
//     tile; a second tcgen05.mma gives the next layer's messages z = h Pi;
//   * the last layer forms y = h D + d in the epilogue instead.
// The operand tile and the accumulators are double-buffered, so the
// aggregation of one tile overlaps the MMAs and the epilogue of the one
// before.  Before the layers, eight lanes per particle write the edge records
// (the four weights of every pair closer than 2h, FP16, with the neighbour
// index), and the first layer launch forms the input layer h_0 = relu(x W_in
// + b_in) and z_0.
//
// Operand layout in shared memory (K-major, no swizzle): a matrix of R rows
// and K columns is stored as K/8 blocks of R x 16 bytes, block b holding
// columns 8b .. 8b+7 of every row, row r at byte 16 r of its block; in the
// tcgen05 shared-memory descriptor the leading-dimension byte offset (between
// blocks adjacent in K) is the block size and the stride-dimension byte
// offset (between 8-row groups) is 128.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sph_mpnn.cuh"

namespace mpnn {

namespace {

// ---------------------------------------------------------------------------
// inline-PTX wrappers: mbarrier, bulk copies, TMA, tcgen05
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity to complete; gives up after about
// one second (false).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16), completing bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// 2D tiled TMA load of one box at (x, y) of the tensor map.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Tensor-memory allocation of ncols columns (a power of two >= 32) by one
// whole warp; the address lands in shared memory at slot.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start address,
// leading- and stride-dimension byte offsets (all >> 4), version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3
// at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) = A B^T (+ D when acc): one tcgen05.mma, issued by one
// thread.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrives on the mbarrier once every tcgen05.mma issued so far by this thread
// has completed.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's lane (32x32b
// shape: warp w reads lanes 32 (w % 4) .. +31).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float2 unpack2(uint32_t u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}

__device__ __forceinline__ float2 unpack_h2(uint32_t u) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// ---------------------------------------------------------------------------
// roles and shared-memory plan of the layer kernel (bytes from a 1024-aligned
// base).  Warps 0..15 aggregate (or, in the first layer, form h_0), warps
// 16..23 run the epilogue (warp w reads tensor-memory lanes 32 (w % 4) ..
// +31), warp 24 allocates tensor memory and its lane 0 issues the TMA loads
// and the tcgen05.mma; the operand tile and the accumulators are double
// buffered, so the aggregation of one tile overlaps the MMAs and epilogue of
// the one before.
// ---------------------------------------------------------------------------
constexpr int TC_AGG_WARPS = 16, TC_EPI_WARPS = 8;
constexpr int TC_CTL_WARP = TC_AGG_WARPS + TC_EPI_WARPS;
constexpr int TC_THREADS = 32 * (TC_CTL_WARP + 1);
constexpr uint32_t BLK_A = TC_M * 16;                  // one 8-column block of 128 rows
constexpr uint32_t BLK_PI = MP_P * 16;                 // one 8-column block of Pi^T (32 rows)
constexpr uint32_t A_BYTES = (MP_CAT / 8) * BLK_A;     // one operand tile [h, g]
constexpr uint32_t SM_BU = 0;                          // U_l^T image, 32 blocks
constexpr uint32_t SM_A = SM_BU + (uint32_t)TC_U_BYTES;   // two operand tiles
constexpr uint32_t SM_BPI = SM_A + 2 * A_BYTES;        // Pi^T image, 16 blocks
constexpr uint32_t SM_PAR = SM_BPI + (uint32_t)TC_PI_BYTES;   // FP32 parameters
constexpr uint32_t SM_BAR = SM_PAR + 4096;             // mbarriers, then the TMEM address
constexpr uint32_t SM_TOTAL = SM_BAR + 256;
constexpr size_t SM_REQUEST = SM_TOTAL + 1024;         // + alignment of the base
static_assert(SM_REQUEST <= 227 * 1024, "shared memory per CTA");
static_assert(TC_U_BYTES == 32 * BLK_A && TC_PI_BYTES == 16 * BLK_PI, "weight image sizes");
static_assert(TC_AGG_WARPS * 32 == TC_M * 4, "one aggregation pass of 4 lanes per row");

// Tensor memory: the U accumulators of the two buffers at columns 0 and 128,
// the message accumulators at 256 and 288.
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TMEM_Z = 256;

enum TcMode { TC_FIRST = 0, TC_MID = 1, TC_LAST = 2 };

// BF16 images: u_img[l] (n, k) = U_l[k][n] at element (k / 8) * 1024 + 8 n +
// k % 8; pi_img[l] (n, k) = Pi_l[k][n] at (k / 8) * 256 + 8 n + k % 8.
struct ImageOffsets {
    long long U[MP_L], Pi[MP_L];
};

__global__ void k_weight_images(const float *__restrict__ param, ImageOffsets off,
                                __nv_bfloat16 *__restrict__ u_img,
                                __nv_bfloat16 *__restrict__ pi_img) {
    const int per_u = MP_H * MP_CAT, per_pi = MP_P * MP_H;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < MP_L * per_u) {
        int l = t / per_u, e = t % per_u;
        int kb = e / (8 * MP_H), n = (e / 8) % MP_H, k = 8 * kb + e % 8;
        u_img[t] = __float2bfloat16_rn(param[off.U[l] + (long long)k * MP_H + n]);
        return;
    }
    t -= MP_L * per_u;
    if (t < MP_L * per_pi) {
        int l = t / per_pi, e = t % per_pi;
        int kb = e / (8 * MP_P), n = (e / 8) % MP_P, k = 8 * kb + e % 8;
        pi_img[t] = __float2bfloat16_rn(param[off.Pi[l] + (long long)k * MP_P + n]);
    }
}

struct TcArgs {
    PhysT<float> P;
    Hot<float> hot;
    Csf<float> csf;
    NList nl;
    int n;
    float inv_uref;
    const float *param;
    long long off0, off1;           // parameter offsets: W_in (FIRST) or c_l; D (LAST)
    const __nv_bfloat16 *u_img;     // this layer's U^T image (MID, LAST)
    const __nv_bfloat16 *pi_img;    // the next messages' Pi^T image (FIRST, MID)
    uint4 *edge;
    unsigned *ecnt;
    __nv_bfloat16 *h;
    const __nv_bfloat16 *zin;
    __nv_bfloat16 *zout;
    float2 *y;
    unsigned *err;
    int stall;                      // test hook: issue no operand loads
};

// Edge records of particle a: every pair closer than 2h as {b, (w0, w1),
// (w2, w3), 0} with FP16 weights (the pairs of Sec. 2-7; the network's edge
// weights), padded with zero-weight records pointing at a itself to a
// multiple of eight.  Eight lanes per particle (four particles per warp), lane
// j taking list entries j, j + 8, ...; the records of one pass keep the list
// order.
template <int K>
__global__ void __launch_bounds__(256) k_tc_edges(PhysT<float> P, Hot<float> hot, NList nl, int n,
                                                  float inv_uref, uint4 *__restrict__ edge,
                                                  unsigned *__restrict__ ecnt) {
    const unsigned lane = threadIdx.x & 31u, j = lane & 7u, gbit = lane & 24u;
    const unsigned a = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool live = a < (unsigned)n;
    const unsigned cnt = live ? nl.cnt[a] : 0u;
    const unsigned cmax = __reduce_max_sync(0xffffffffu, cnt);
    const uint32_t *__restrict__ e = nl.e + (size_t)(live ? a : 0u) * LIST_SLOTS;
    uint4 *__restrict__ out = edge + (size_t)(live ? a : 0u) * LIST_SLOTS;
    V4f ha{};
    if (live) ha = hot.H0[a];
    unsigned outc = 0;
    for (unsigned base = 0; base < cmax; base += 8) {
        unsigned k = base + j, o = 0;
        EdgeW ew{};
        bool ok = false;
        if (k < cnt) {
            float rx, ry, r2, du, dv;
            ok = list_pair(P, hot, e, k, a, ha, o, rx, ry, r2, du, dv);
            if (ok) ew = edge_weights<K>(P, rx, ry, r2, du, dv, hot.H1[o].x, inv_uref);
        }
        const unsigned m = (__ballot_sync(0xffffffffu, ok) >> gbit) & 0xFFu;
        if (ok) {
            unsigned slot = outc + __popc(m & ((1u << j) - 1u));
            out[slot] = make_uint4(o, pack_h2(ew.w[0], ew.w[1]), pack_h2(ew.w[2], ew.w[3]), 0u);
        }
        outc += __popc(m);
    }
    if (!live) return;
    const unsigned c8 = (outc + 7u) & ~7u;      // <= LIST_SLOTS, a multiple of 8
    if (j < c8 - outc) out[outc + j] = make_uint4(a, 0u, 0u, 0u);
    if (j == 0) ecnt[a] = c8;
}

// Node inputs of particle a (as k_mp_inputs): 100 (rho/rho0 - 1), N_a,
// C_a, h |n_a|.
__device__ __forceinline__ void node_inputs(const TcArgs &A, unsigned a, float (&x)[4]) {
    V4f h1 = A.hot.H1[a];
    V2f nh = A.csf.nhat[a];
    V2f nv = A.csf.nvec[a];
    x[0] = 100.0f * (h1.y / A.P.rho0 - 1.0f);
    x[1] = (nh.x != 0.0f || nh.y != 0.0f) ? 1.0f : 0.0f;
    x[2] = A.csf.C[a];
    x[3] = A.P.h * sqrtf(nv.x * nv.x + nv.y * nv.y);
}

// Messages of row a of the tile, channels 8j .. 8j+7 (j = lane % 4), all
// four weights: acc[k][i] = sum_b w_k,ab z_b[8j + i] over the edge records.
// The four lanes of a row hold eight records at a time (two each; the next
// eight load while these are used) and pass them round by shuffles; every
// lane of the warp takes part until the longest of its eight rows is done
// (rows past n, and rows that finished, add zero-weight records of particle
// `self`).
__device__ __forceinline__ void aggregate(const TcArgs &A, unsigned a, bool live, unsigned lane,
                                          float (&acc)[4][8]) {
    const unsigned j = lane & 3u, g0 = lane & ~3u;
    const unsigned self = live ? a : 0u;
    const uint4 *__restrict__ E = A.edge + (size_t)self * LIST_SLOTS;
    // the first records load beside the count (slots past the count hold
    // stale records and are replaced by pad below)
    const uint4 f0 = __ldg(E + j), f1 = __ldg(E + 4 + j);
    const unsigned c8 = live ? A.ecnt[a] : 0u;
    const unsigned cmax = __reduce_max_sync(0xffffffffu, c8);
    const __nv_bfloat16 *__restrict__ z = A.zin + 8 * j;
    const uint4 pad = make_uint4(self, 0u, 0u, 0u);
    uint4 cur[2] = {c8 > 0 ? f0 : pad, c8 > 0 ? f1 : pad};
    for (unsigned e = 0; e < cmax; e += 8) {
        const bool more = e + 8 < c8;
        // slots clamped into the row so that the loads need no branch
        const unsigned s0 = min(e + 8 + j, (unsigned)LIST_SLOTS - 8), s1 = s0 + 4;
        const uint4 l0 = __ldg(E + s0), l1 = __ldg(E + s1);
        const uint4 nxt[2] = {more ? l0 : pad, more ? l1 : pad};
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint4 zz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                unsigned idx = __shfl_sync(0xffffffffu, cur[half].x, g0 + u);
                if (index_bad(A.P, idx)) idx = self;
                zz[u] = __ldg(reinterpret_cast<const uint4 *>(z + (size_t)idx * MP_P));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 w01 = unpack_h2(__shfl_sync(0xffffffffu, cur[half].y, g0 + u));
                const float2 w23 = unpack_h2(__shfl_sync(0xffffffffu, cur[half].z, g0 + u));
                const float w[4] = {w01.x, w01.y, w23.x, w23.y};
                const uint32_t zw[4] = {zz[u].x, zz[u].y, zz[u].z, zz[u].w};
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float2 zp = unpack2(zw[p]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        acc[k][2 * p] = fmaf(w[k], zp.x, acc[k][2 * p]);
                        acc[k][2 * p + 1] = fmaf(w[k], zp.y, acc[k][2 * p + 1]);
                    }
                }
            }
        }
        cur[0] = nxt[0];
        cur[1] = nxt[1];
    }
}

// Stores 16 BF16 values (8 packed words) as two 16-byte pieces.
__device__ __forceinline__ void store16(void *p0, void *p1, const uint32_t (&pk)[8]) {
    *reinterpret_cast<uint4 *>(p0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4 *>(p1) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One layer of the inference pass (MODE: TC_FIRST, TC_MID or TC_LAST), one
// persistent CTA per SM over the tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...; hmap: the TMA map of the hidden state h (n rows of 128 BF16; boxes of
// 8 columns x 128 rows, rows past n read as zeros).  The i-th tile of a CTA
// uses buffer b = i % 2; the mbarriers of buffer b complete once per tile
// that uses it (parity (i / 2) % 2):
//   full[b]  the operand tile is in place: 16 aggregation warps + the
//            control thread's arrival (with the TMA bytes of h);
//   acc[b]   the U accumulator is complete (tcgen05.commit);
//   hnew[b]  the epilogue wrote h_{l+1} into the tile (8 warps);
//   zf[b]    the message accumulator is complete (tcgen05.commit);
//   free[b]  the epilogue is done with the tile and its tensor memory.
// Every wait gives up after about a second: the error word gets
// ERR_TIMEOUT, the role stops, and the block ends.
template <int MODE, int K>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_layer(const __grid_constant__ CUtensorMap hmap, const TcArgs A) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) &
                                          ~static_cast<uintptr_t>(1023));
    const uint32_t sbase = smem_u32(base);
    const unsigned tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t BAR = sbase + SM_BAR;
    const uint32_t bar_w = BAR;
    auto bar_full = [&](int b) { return BAR + 8u + 8u * b; };
    auto bar_acc = [&](int b) { return BAR + 24u + 8u * b; };
    auto bar_hnew = [&](int b) { return BAR + 40u + 8u * b; };
    auto bar_zf = [&](int b) { return BAR + 56u + 8u * b; };
    auto bar_free = [&](int b) { return BAR + 72u + 8u * b; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + SM_BAR + 128);
    float *par = reinterpret_cast<float *>(base + SM_PAR);
    const int n = A.n, ntiles = (n + TC_M - 1) / TC_M;
    const int my_tiles =
        (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto tile_row0 = [&](int i) { return ((int)blockIdx.x + i * (int)gridDim.x) * TC_M; };
    auto tile_at = [&](int b) { return base + SM_A + b * A_BYTES; };
    auto timeout = [&]() { atomicOr(A.err, (unsigned)ERR_TIMEOUT); };

    if (tid == 0) {
        mbar_init(bar_w, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_full(b), TC_AGG_WARPS + 1);
            mbar_init(bar_acc(b), 1);
            mbar_init(bar_hnew(b), TC_EPI_WARPS);
            mbar_init(bar_zf(b), 1);
            mbar_init(bar_free(b), TC_EPI_WARPS);
        }
        fence_mbar_init();
    }
    if (warp == TC_CTL_WARP) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    // FP32 parameters: W_in and b_in (FIRST; contiguous), c_l (MID, LAST), D
    // and d (LAST; contiguous)
    if (MODE == TC_FIRST) {
        for (int t = tid; t < MP_IN * MP_H + MP_H; t += TC_THREADS) par[t] = A.param[A.off0 + t];
    } else {
        for (int t = tid; t < MP_H; t += TC_THREADS) par[t] = A.param[A.off0 + t];
        if (MODE == TC_LAST)
            for (int t = tid; t < MP_H * MP_OUT + MP_OUT; t += TC_THREADS)
                par[MP_H + t] = A.param[A.off1 + t];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tmem_slot);

    if (warp < TC_AGG_WARPS) {
        // ---- operand producers ------------------------------------------
        for (int i = 0; i < my_tiles; ++i) {
            const int b = i & 1, m0 = tile_row0(i);
            if (i >= 2 && !mbar_wait(bar_free(b), ((i >> 1) - 1) & 1)) {
                timeout();
                break;
            }
            unsigned char *Ab = tile_at(b);
            if (MODE != TC_FIRST) {
                // messages into columns 128..255: four lanes per row
                const unsigned r = tid >> 2, j = tid & 3u, a = (unsigned)m0 + r;
                // the next tile's records (its first 32 slots) on their way to L2
                if (i + 1 < my_tiles) {
                    const unsigned an = (unsigned)tile_row0(i + 1) + r;
                    if (an < (unsigned)n) prefetch_l2(A.edge + (size_t)an * LIST_SLOTS + 8 * j);
                }
                float acc[4][8];
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[k][q] = 0.f;
                aggregate(A, a, a < (unsigned)n, lane, acc);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    // columns 128 + 32k + 8j .. +7: block 16 + 4k + j
                    *reinterpret_cast<uint4 *>(Ab + (16 + 4 * k + j) * BLK_A + r * 16) =
                        make_uint4(pack2(acc[k][0], acc[k][1]), pack2(acc[k][2], acc[k][3]),
                                   pack2(acc[k][4], acc[k][5]), pack2(acc[k][6], acc[k][7]));
                }
            } else {
                // input layer: row r, columns 32 cg .. 32 cg + 31
                const unsigned r = tid & (TC_M - 1), cg = tid >> 7, a = (unsigned)m0 + r;
                const bool live = a < (unsigned)n;
                float x[4] = {0.f, 0.f, 0.f, 0.f};
                if (live) node_inputs(A, a, x);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int c0 = 32 * cg + 16 * half;
                    uint32_t pk[8];
#pragma unroll
                    for (int c = 0; c < 16; c += 2) {
                        float v[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int col = c0 + c + e;
                            float sum = par[MP_IN * MP_H + col];
#pragma unroll
                            for (int q = 0; q < MP_IN; ++q) sum = fmaf(x[q], par[q * MP_H + col], sum);
                            v[e] = live ? fmaxf(sum, 0.f) : 0.f;
                        }
                        pk[c / 2] = pack2(v[0], v[1]);
                    }
                    store16(Ab + (c0 / 8) * BLK_A + r * 16, Ab + (c0 / 8 + 1) * BLK_A + r * 16, pk);
                    if (live) {
                        uint4 *g = reinterpret_cast<uint4 *>(A.h + (size_t)a * MP_H + c0);
                        store16(g, g + 1, pk);
                    }
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full(b));
        }
    } else if (warp < TC_CTL_WARP) {
        // ---- epilogue ---------------------------------------------------
        const unsigned q = warp & 3u, ch = (warp - TC_AGG_WARPS) >> 2, r = 32 * q + lane;
        const uint32_t tl = tmem + ((32 * q) << 16);
        for (int i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            const uint32_t par_u = (uint32_t)(i >> 1) & 1u;
            const unsigned a = (unsigned)tile_row0(i) + r;
            const bool live = a < (unsigned)n;
            unsigned char *Ab = tile_at(b);
            if (MODE != TC_FIRST) {
                // the tile (h_l by TMA) and the U accumulator
                if (!mbar_wait(bar_full(b), par_u) || !mbar_wait(bar_acc(b), par_u)) {
                    timeout();
                    break;
                }
                tc_fence_after();
                // MID: warp halves ch = 0, 1 take columns 0..63 and 64..127;
                // LAST: the ch = 0 warps take all 128 (y needs the whole row)
                float yp0 = 0.f, yp1 = 0.f;
                const int nchunk = MODE == TC_MID ? 4 : (ch == 0 ? 8 : 0);
#pragma unroll 1
                for (int c4 = 0; c4 < nchunk; ++c4) {
                    const int c0 = (MODE == TC_MID ? 64 * ch : 0) + 16 * c4;
                    float v[16];
                    tc_ld16(tl + b * 128 + c0, v);
                    unsigned char *hs0 = Ab + (c0 / 8) * BLK_A + r * 16;
                    unsigned char *hs1 = Ab + (c0 / 8 + 1) * BLK_A + r * 16;
                    const uint4 o0 = *reinterpret_cast<const uint4 *>(hs0);
                    const uint4 o1 = *reinterpret_cast<const uint4 *>(hs1);
                    const uint32_t ow[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
                    float hn[16];
#pragma unroll
                    for (int c = 0; c < 16; c += 2) {
                        const float2 ho = unpack2(ow[c / 2]);
                        hn[c] = ho.x + fmaxf(v[c] + par[c0 + c], 0.f);
                        hn[c + 1] = ho.y + fmaxf(v[c + 1] + par[c0 + c + 1], 0.f);
                    }
                    if (MODE == TC_MID) {
                        uint32_t pk[8];
#pragma unroll
                        for (int c = 0; c < 16; c += 2) pk[c / 2] = pack2(hn[c], hn[c + 1]);
                        store16(hs0, hs1, pk);
                        if (live) {
                            uint4 *g = reinterpret_cast<uint4 *>(A.h + (size_t)a * MP_H + c0);
                            store16(g, g + 1, pk);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            yp0 = fmaf(hn[c], par[MP_H + 2 * (c0 + c)], yp0);
                            yp1 = fmaf(hn[c], par[MP_H + 2 * (c0 + c) + 1], yp1);
                        }
                    }
                }
                if (MODE == TC_MID) {
                    fence_async_smem();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_hnew(b));
                } else {
                    // y = h D + d
                    if (ch == 0 && live)
                        A.y[a] = make_float2(par[MP_H + MP_H * MP_OUT] + yp0,
                                             par[MP_H + MP_H * MP_OUT + 1] + yp1);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_free(b));
                    continue;
                }
            }
            // the messages z = h Pi of this tile: columns 16 ch .. 16 ch + 15
            if (!mbar_wait(bar_zf(b), par_u)) {
                timeout();
                break;
            }
            tc_fence_after();
            float v[16];
            tc_ld16(tl + TMEM_Z + 32 * b + 16 * ch, v);
            if (live) {
                uint32_t pk[8];
#pragma unroll
                for (int c = 0; c < 16; c += 2) pk[c / 2] = pack2(v[c], v[c + 1]);
                uint4 *g = reinterpret_cast<uint4 *>(A.zout + (size_t)a * MP_P + 16 * ch);
                store16(g, g + 1, pk);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_free(b));
        }
    } else if (lane == 0) {
        // ---- control: weights, TMA loads, tcgen05.mma --------------------
        bool ok = true;
        uint32_t pend_bar = 0, pend_par = 0;   // the last commit, for a drain on failure
        mbar_expect_tx(bar_w, (MODE != TC_FIRST ? (uint32_t)TC_U_BYTES : 0u) +
                                  (MODE != TC_LAST ? (uint32_t)TC_PI_BYTES : 0u));
        if (MODE != TC_FIRST) bulk_g2s(sbase + SM_BU, A.u_img, (uint32_t)TC_U_BYTES, bar_w);
        if (MODE != TC_LAST) bulk_g2s(sbase + SM_BPI, A.pi_img, (uint32_t)TC_PI_BYTES, bar_w);
        if (!mbar_wait(bar_w, 0)) {
            timeout();
            ok = false;
        }
        auto load = [&](int i) {
            const int b = i & 1;
            if (MODE != TC_FIRST) {
                mbar_expect_tx(bar_full(b), (uint32_t)(TC_M * MP_H * 2));
                const uint32_t dst = sbase + SM_A + b * A_BYTES;
                for (int blk = 0; blk < MP_H / 8; ++blk)
                    tma_load_2d(dst + blk * BLK_A, &hmap, 8 * blk, tile_row0(i), bar_full(b));
            } else {
                mbar_arrive(bar_full(b));
            }
        };
        for (int i = 0; ok && !A.stall && i < my_tiles && i < 2; ++i) load(i);
        for (int i = 0; ok && i < my_tiles; ++i) {
            const int b = i & 1;
            const uint32_t par_u = (uint32_t)(i >> 1) & 1u;
            const uint32_t at = sbase + SM_A + b * A_BYTES;
            if (!mbar_wait(bar_full(b), par_u)) {
                ok = false;
                break;
            }
            tc_fence_after();
            if (MODE != TC_FIRST) {
                // acc = [h, g] U_l (K = 256 in 16 steps)
#pragma unroll 1
                for (int ks = 0; ks < MP_CAT / 16; ++ks)
                    tc_mma(tmem + b * 128, smem_desc(at + 2 * ks * BLK_A, BLK_A, 128),
                           smem_desc(sbase + SM_BU + 2 * ks * BLK_A, BLK_A, 128),
                           idesc_bf16(TC_M, MP_H), ks > 0 ? 1u : 0u);
                tc_commit(bar_acc(b));
                pend_bar = bar_acc(b);
                pend_par = par_u;
            }
            if (MODE != TC_LAST) {
                if (MODE == TC_MID) {
                    if (!mbar_wait(bar_hnew(b), par_u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                // z = h Pi (K = 128 in 8 steps, N = 32)
#pragma unroll 1
                for (int ks = 0; ks < MP_H / 16; ++ks)
                    tc_mma(tmem + TMEM_Z + 32 * b, smem_desc(at + 2 * ks * BLK_A, BLK_A, 128),
                           smem_desc(sbase + SM_BPI + 2 * ks * BLK_PI, BLK_PI, 128),
                           idesc_bf16(TC_M, MP_P), ks > 0 ? 1u : 0u);
                tc_commit(bar_zf(b));
                pend_bar = bar_zf(b);
                pend_par = par_u;
            }
            if (i + 2 < my_tiles) {
                if (!mbar_wait(bar_free(b), par_u)) {
                    ok = false;
                    break;
                }
                load(i + 2);
            }
        }
        if (!ok) {
            timeout();
            if (pend_bar) mbar_wait(pend_bar, pend_par);   // let the last MMAs finish
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == TC_CTL_WARP) tmem_dealloc(tmem, TMEM_COLS);
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point
// query, so the library links no driver stub).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

template <int MODE, int K>
cudaError_t launch_layer(int grid, const CUtensorMap &hmap, const TcArgs &A, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_layer<MODE, K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_REQUEST);
    if (e != cudaSuccess) return e;
    k_tc_layer<MODE, K><<<grid, TC_THREADS, SM_REQUEST, s>>>(hmap, A);
    return cudaGetLastError();
}

template <int K>
cudaError_t forward_k(int grid, const CUtensorMap &hmap, TcArgs A, const __nv_bfloat16 *u_img,
                      const __nv_bfloat16 *pi_img, const MpScratch &scr, cudaStream_t s) {
    constexpr size_t U_EL = TC_U_BYTES / 2, PI_EL = TC_PI_BYTES / 2;
    A.pi_img = pi_img;
    A.zout = scr.z[0];
    A.off0 = kMP.W_in;
    k_tc_edges<K><<<(A.n + 31) / 32, 256, 0, s>>>(A.P, A.hot, A.nl, A.n, A.inv_uref, A.edge, A.ecnt);
    cudaError_t e = launch_layer<TC_FIRST, K>(grid, hmap, A, s);
    for (int l = 0; l < MP_L && e == cudaSuccess; ++l) {
        A.off0 = kMP.c[l];
        A.off1 = kMP.D;
        A.u_img = u_img + l * U_EL;
        A.zin = scr.z[l & 1];
        if (l + 1 < MP_L) {
            A.pi_img = pi_img + (l + 1) * PI_EL;
            A.zout = scr.z[(l + 1) & 1];
            e = launch_layer<TC_MID, K>(grid, hmap, A, s);
        } else {
            e = launch_layer<TC_LAST, K>(grid, hmap, A, s);
        }
    }
    return e;
}

}  // namespace

void tc_weight_images(const float *param, __nv_bfloat16 *u_img, __nv_bfloat16 *pi_img,
                      cudaStream_t s) {
    const int total = MP_L * (MP_H * MP_CAT + MP_P * MP_H);
    ImageOffsets off;
    for (int l = 0; l < MP_L; ++l) {
        off.U[l] = kMP.U[l];
        off.Pi[l] = kMP.Pi[l];
    }
    k_weight_images<<<(total + 255) / 256, 256, 0, s>>>(param, off, u_img, pi_img);
}

cudaError_t tc_forward(const CtxView &v, float inv_uref, const float *param,
                       const __nv_bfloat16 *u_img, const __nv_bfloat16 *pi_img,
                       const MpScratch &scr, unsigned *err, int stall) {
    if (v.n <= 0) return cudaSuccess;
    if (v.n > scr.cap) return cudaErrorInvalidValue;
    EncodeTiled enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap hmap;
    const cuuint64_t dims[2] = {(cuuint64_t)MP_H, (cuuint64_t)v.n};
    const cuuint64_t strides[1] = {(cuuint64_t)MP_H * 2};
    const cuuint32_t box[2] = {8u, (cuuint32_t)TC_M};
    const cuuint32_t estr[2] = {1u, 1u};
    if (enc(&hmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, scr.h, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, v.device);
    if (e != cudaSuccess) return e;
    const int ntiles = (v.n + TC_M - 1) / TC_M;
    const int grid = ntiles < sms ? ntiles : sms;
    TcArgs A{};
    A.P = v.P;
    A.hot = v.hot;
    A.csf = v.csf;
    A.nl = v.nl;
    A.n = v.n;
    A.inv_uref = inv_uref;
    A.param = param;
    A.edge = scr.edge;
    A.ecnt = scr.ecnt;
    A.h = scr.h;
    A.y = scr.y;
    A.err = err;
    A.stall = stall;
    if (v.P.kernel == 1) return forward_k<1>(grid, hmap, A, u_img, pi_img, scr, v.stream);
    return forward_k<0>(grid, hmap, A, u_img, pi_img, scr, v.stream);
}

}  // namespace mpnn
