// Definitions shared by the two halves of the learned surrogate: the
// network's shape and parameter layout, and the edge weights it reads from
// the SPH neighbour lists (sph_mpnn.cu: FP32 training and reference forward;
// sph_mpnn_tc.cu: the tensor-core inference pass).
#pragma once

#include <cuda_bf16.h>

#include "sph_device.cuh"

namespace mpnn {

using namespace sph;

using V4f = Vec<float>::v4;
using V2f = Vec<float>::v2;

constexpr int MP_IN = 4, MP_H = 128, MP_P = 32, MP_L = 3, MP_OUT = 2;
constexpr int MP_G = 4 * MP_P;        // aggregated features per particle
constexpr int MP_CAT = MP_H + MP_G;   // input width of the update layers

// Offsets (in floats) of the packed parameters: W_in, b_in, then per layer
// Pi_l, U_l, c_l, then D, d; every matrix row-major (fan-in x fan-out).
struct Layout {
    long long W_in, b_in, Pi[MP_L], U[MP_L], c[MP_L], D, d, total;
};

constexpr Layout make_layout() {
    Layout L{};
    long long o = 0;
    L.W_in = o; o += MP_IN * MP_H;
    L.b_in = o; o += MP_H;
    for (int l = 0; l < MP_L; ++l) {
        L.Pi[l] = o; o += MP_H * MP_P;
        L.U[l] = o; o += MP_CAT * MP_H;
        L.c[l] = o; o += MP_H;
    }
    L.D = o; o += MP_H * MP_OUT;
    L.d = o; o += MP_OUT;
    L.total = o;
    return L;
}

constexpr Layout kMP = make_layout();

// ---------------------------------------------------------------------------
// edge weights
// ---------------------------------------------------------------------------
struct EdgeW {
    float w[4];
};

// Weights of the ordered pair (s, o) seen from particle s ("self") and its
// list entry o: rx, ry = r_s - r_o; du, dv = u_s - u_o; V the volume of the
// particle whose feature is summed (o in the forward sum over s's list).
template <int K>
__device__ __forceinline__ EdgeW edge_weights(const PhysT<float> &P, float rx, float ry, float r2,
                                              float du, float dv, float V, float inv_uref) {
    float q, iq, ri;
    q_of(r2, P.h, P.inv_h, q, iq, ri);
    float W = kernel_W<float, K>(P, q);
    float F = kernel_F<float, K>(P, q, iq);
    float VF = V * F * P.h;
    EdgeW e;
    e.w[0] = V * W;
    e.w[1] = VF * rx;
    e.w[2] = VF * ry;
    e.w[3] = VF * (du * rx + dv * ry) * inv_uref;
    return e;
}

// Entry k of particle s's list: returns false unless it is a pair closer than
// 2h (the same FP32 band + exact FP64 test as the SPH sweeps); fills the
// neighbour index and the self-minus-neighbour offsets and velocities.
__device__ __forceinline__ bool list_pair(const PhysT<float> &P, const Hot<float> &hot,
                                          const uint32_t *__restrict__ e, unsigned k, unsigned s,
                                          const V4f &hs, unsigned &o, float &rx, float &ry,
                                          float &r2, float &du, float &dv) {
    uint32_t ent = e[k];
    o = ent & 0x0FFFFFFFu;
    if (index_bad(P, o)) return false;
    V4f ho = hot.H0[o];
    rx = off_diff<float>(P, hs.x, ho.x, code_cells((ent >> 28) & 3u));
    ry = off_diff<float>(P, hs.y, ho.y, code_cells(ent >> 30));
    r2 = rx * rx + ry * ry;
    if (r2 >= P.H2hi) return false;
    if (r2 >= P.H2lo && !exact_within(hot.pos[s], hot.pos[o], P.H2d)) return false;
    du = hs.z - ho.z;
    dv = hs.w - ho.w;
    return true;
}


// ---------------------------------------------------------------------------
// tensor-core inference (sph_mpnn_tc.cu)
// ---------------------------------------------------------------------------
// Rows of one tile of the inference pass (the M of each tcgen05.mma).
constexpr int TC_M = 128;

// Sizes of the BF16 weight images of one layer, laid out as the shared-memory
// operand of tcgen05.mma (sph_mpnn_tc.cu): U_l^T (128 x 256) and Pi_l^T (32 x
// 128) in 8-column core-matrix blocks.
constexpr size_t TC_U_BYTES = (size_t)MP_H * MP_CAT * 2;
constexpr size_t TC_PI_BYTES = (size_t)MP_P * MP_H * 2;

// Per-pass scratch of the inference pass, capacity rows each.
struct MpScratch {
    uint4 *edge = nullptr;          // LIST_SLOTS edge records per particle
    unsigned *ecnt = nullptr;       // records per particle (a multiple of 8)
    __nv_bfloat16 *h = nullptr;     // hidden state, MP_H per particle
    __nv_bfloat16 *z[2] = {};       // messages, MP_P per particle (ping-pong)
    float2 *y = nullptr;            // output
    long long cap = 0;
};

// BF16 images of U_l^T and Pi_l^T (l < MP_L) from the FP32 parameters.
void tc_weight_images(const float *param, __nv_bfloat16 *u_img, __nv_bfloat16 *pi_img,
                      cudaStream_t s);

// The inference pass over the view's n particles: y = network(state) into
// scr.y.  Five launches: the edge records, the input layer with the first
// messages, the three message-passing layers.  err (the context's sticky
// error word) receives ERR_TIMEOUT if a bounded wait ran out.
// stall != 0: the test hook of sph_mpnn_inject_stall (no operand loads).
cudaError_t tc_forward(const CtxView &v, float inv_uref, const float *param,
                       const __nv_bfloat16 *u_img, const __nv_bfloat16 *pi_img,
                       const MpScratch &scr, unsigned *err, int stall = 0);

}  // namespace mpnn
