// api.cu -- the C ABI of include/jacpcg.h: contexts, the device workspace
// arena, plans (instance tables + tile lists + workspace on the device),
// CUDA-graph capture and the launch sequence Gram -> iteration -> W = H X
// -> finalise for every K class of a (possibly ragged) batch.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <array>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/jacpcg.h"
#include "common.cuh"
#include "kernels.h"

using namespace jacpcg;

namespace {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x, size_t a = ALIGN) { return (x + a - 1) / a * a; }

int k_class(int K) {
    int c = 8;
    while (c < K) c <<= 1;
    return c;
}

// ---------------------------------------------------------------------------
// First-fit allocator over one device buffer, with stream-ordered release:
// a block freed while kernels may still read it is parked with an event and
// returned once the event has completed.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
    struct Pending {
        size_t off, bytes;
        cudaEvent_t ev;
    };
    std::vector<Pending> pending;

    size_t free_bytes() const {
        size_t s = 0;
        for (auto &kv : free_) s += kv.second;
        return s;
    }
    void insert_free(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    void reap(bool wait_one) {
        for (size_t i = 0; i < pending.size();) {
            cudaError_t q = wait_one && i == 0 ? cudaEventSynchronize(pending[i].ev)
                                               : cudaEventQuery(pending[i].ev);
            if (q == cudaSuccess) {
                insert_free(pending[i].off, pending[i].bytes);
                cudaEventDestroy(pending[i].ev);
                pending.erase(pending.begin() + i);
                wait_one = false;
            } else {
                if (q != cudaErrorNotReady) (void)cudaGetLastError();
                ++i;
            }
        }
    }
    bool try_alloc(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t o = it->first;
                free_.erase(it);
                if (rest) free_.emplace(o + bytes, rest);
                return true;
            }
        }
        return false;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = align_up(bytes);
        reap(false);
        if (try_alloc(bytes, off)) return true;
        while (!pending.empty()) {
            reap(true);
            if (try_alloc(bytes, off)) return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes, cudaEvent_t ev) {
        bytes = align_up(bytes);
        if (ev) pending.push_back({off, bytes, ev});
        else insert_free(off, bytes);
    }
};

// What one kernel launch of a plan covers.
struct Launch {
    enum Kind {
        GRAM, PCG, HX, GRAM_TC, GRAM_TCX, HX_TC, HX_TCW, PCG_TC, CHOL, SINR, TCW_PREP, PCG_TCW, GRAM_BF16, HX_BF16,
        RESID_TC
    } kind;
    int phase;        // 0 Gram, 1 iteration, 2 W = H X, 3 SINR (after the power factor), 4 refinement
    int param;        // TB (Gram), KC (iteration), TN (W = H X)
    size_t list_off;  // byte offset of its work list inside the plan block
    int count;        // CTAs
    int shape = 0;    // iteration launch shape (index into PCG_SHAPES)
    size_t list2_off = 0;   // RESID_TC: its (instance, column) jobs; list_off / count: the instances
    int count2 = 0;
};

}  // namespace

struct jacpcg_ctx {
    jacpcg_config cfg{};
    Arena arena;
    bool broken = false;
    cudaError_t last_error = cudaSuccess;   // first CUDA error that broke the context
    int64_t launches = 0;
    // pinned staging for asynchronous table uploads of jacpcg_precode
    char *staging = nullptr;
    size_t staging_bytes = 0;
    cudaEvent_t staging_ev = nullptr;
    bool staging_pending = false;
    cudaStream_t capture_stream = nullptr;   // graphs are captured here, launched on the caller's
    // per-phase events of the profiled executes since the last read
    std::vector<std::array<cudaEvent_t, 5>> prof_pool;
    size_t prof_used = 0;
    int last_launches = 0;
    std::vector<jacpcg_plan *> plans;
    // chosen iteration per K class: -1 the tensor-core kernel where the class,
    // precision and variant allow it (else SIMT shape 0), 0.. a SIMT launch shape
    int pcg_shape_idx[6] = {-1, -1, -1, -1, -1, -1};
    CUtensorMap amap{};   // the arena as rows of 64 floats, for the tiled copies of A
    void *encode = nullptr;   // the driver's tensor-map encoder (cuTensorMapEncodeTiled)
};

struct jacpcg_plan {
    jacpcg_ctx *ctx = nullptr;
    size_t off = 0, bytes = 0;
    char *dev = nullptr;
    int n_inst = 0;
    DevInst *d_insts = nullptr;
    DevAccum acc{};
    DevOut out{};
    std::vector<Launch> launches;
    int use_graph = 0;
    cudaGraphExec_t gexec = nullptr;
    int graph_launches = 0;
    cudaEvent_t done = nullptr;
    bool executed = false;
    int refine_sweeps = 0;
    bool want_hist = false;       // some instance asked for its refinement residual history
    size_t res_off = 0;
    int n_res = 0;
    int n_rtc = 0;                // instances on the sliced tensor-core residual
    size_t acc_reset_bytes = 0;   // > 0: clear the accumulators before the Gram (multi-job instances)
    size_t tmap_off = 0;          // tensor maps over the bfloat16 channels' H
};

namespace {

jacpcg_status cuda_fail(jacpcg_ctx *ctx, cudaError_t e = cudaErrorUnknown) {
    if (ctx) {
        if (!ctx->broken) ctx->last_error = e;
        ctx->broken = true;
    }
    return JACPCG_ECUDA;
}
#define CK(call)                                   \
    do {                                           \
        const cudaError_t ck_e = (call);           \
        if (ck_e != cudaSuccess) return cuda_fail(ctx, ck_e); \
    } while (0)

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

jacpcg_status validate(const jacpcg_ctx *ctx, const jacpcg_instance *inst, int n) {
    if (!ctx || !inst || n < 1 || n > ctx->cfg.max_instances) return JACPCG_EINVAL;
    for (int i = 0; i < n; ++i) {
        const jacpcg_instance &q = inst[i];
        if (q.K < 1 || q.K > ctx->cfg.max_K || q.M < 1 || q.M > ctx->cfg.max_M) return JACPCG_EINVAL;
        if (q.ldh < q.M || q.ldw < q.M || (q.ldh & 1) || (q.ldw & 1)) return JACPCG_EINVAL;
        if (!q.H || !q.W || !aligned16(q.H) || !aligned16(q.W)) return JACPCG_EINVAL;
        if ((q.X && !aligned16(q.X)) || (q.A && !aligned16(q.A))) return JACPCG_EINVAL;
        if (!std::isfinite(q.xi) || q.xi < 0.0 || (q.K > q.M && !(q.xi > 0.0))) return JACPCG_EINVAL;
        if (!std::isfinite(q.power) || !std::isfinite(q.tol)) return JACPCG_EINVAL;
        if (q.max_iter < 0 || q.max_iter > 4096) return JACPCG_EINVAL;
        if (q.h_dtype != JACPCG_H_C64 && q.h_dtype != JACPCG_H_BF16) return JACPCG_EINVAL;
        if (q.h_dtype == JACPCG_H_BF16 && (q.ldh & 3)) return JACPCG_EINVAL;   // 16-byte columns
        if (q.B && (q.n_rhs < 1 || q.n_rhs > k_class(q.K) || q.ldb < q.K || !aligned16(q.B)))
            return JACPCG_EINVAL;
        if (q.X0 && !aligned16(q.X0)) return JACPCG_EINVAL;
        if (!(q.omega >= 0.f) || !(q.omega < 2.f)) return JACPCG_EINVAL;   // also NaN
        if (q.sinr && (q.B || (reinterpret_cast<uintptr_t>(q.sinr) & 3))) return JACPCG_EINVAL;
        if (!(q.noise >= 0.f) || !std::isfinite(q.noise)) return JACPCG_EINVAL;
    }
    return JACPCG_OK;
}

// right-hand sides of an instance: K for B = I, else n_rhs
int n_cols(const jacpcg_instance &q) { return q.B ? q.n_rhs : q.K; }

// Byte layout of one plan block.
struct Layout {
    size_t insts, gram, tcl, gdl, gxl, pcg, hx, hxl, hwl, res, sinr, twl, twj, tmaps, gbl, hbl, accum, ws, total;
    int n_gram, n_pcg, n_hx, n_res, n_gd, n_gx, n_hw, n_sinr, n_twj, n_tm, n_gb, n_hb, n_rtl, n_rtj;
    size_t rtl, rtj;
    bool refine;
    std::vector<size_t> ws_off;   // per instance
};

int n_wtiles(const jacpcg_instance &q) {
    const int KC = k_class(q.K), TN = hx_tn(KC);
    return ((q.M + HX_TM - 1) / HX_TM) * ((n_cols(q) + TN - 1) / TN);
}
int n_gtiles(const jacpcg_instance &q) {
    const int KC = k_class(q.K), TB = gram_tb(KC);
    const int nb = std::max(1, KC / TB);   // cover the zero padding up to KC as well
    return nb * (nb + 1) / 2;
}
int n_pblocks(const jacpcg_instance &q, const int *shape_idx) {
    const int KC = k_class(q.K);
    const PcgShape s = pcg_shape(KC, shape_idx[kc_index(KC)]);
    const int per = s.CW * s.NW;
    return (n_cols(q) + per - 1) / per;
}
// bfloat16 channels of the 128 and 256 classes: the Gram and W = H X read H
// through tiled tensor copies and run kind::f16 MMAs (gram_bf16.cu,
// hx_bf16.cu); W = H X in jobs of 32 output columns, one ||W||^2 partial per
// 64 antennas and job
bool bf16_native(int precision, const jacpcg_instance &q) {
    return precision == JACPCG_TF32X3 && q.h_dtype == JACPCG_H_BF16 && k_class(q.K) >= 128;
}
int hx_bf16_groups(const jacpcg_instance &q) { return (n_cols(q) + 31) / 32; }
int hx_bf16_slots(const jacpcg_instance &q) { return ((q.M + 63) / 64) * hx_bf16_groups(q); }
size_t wpart_slots(const jacpcg_instance &q) { return std::max(n_wtiles(q), hx_bf16_slots(q)); }
// A, X, 1/diag, W partials; then R and its column norms for refinement; then,
// for the 128 and 256 classes' tensor-core iteration, A as its streamed FP16
// stages (head and tail of real and imaginary parts: 8 KC^2 bytes)
// (and, for the sliced tensor-core residual, A's slices and their row exponents)
size_t inst_ws_bytes(const jacpcg_instance &q, bool refine, bool tcw, bool sliced = false) {
    const size_t KC = k_class(q.K);
    size_t b = align_up(KC * KC * sizeof(float2)) * 2 + align_up(KC * sizeof(float)) +
               align_up(wpart_slots(q) * sizeof(float));
    if (refine) b += align_up(KC * KC * sizeof(float2)) + align_up((2 * KC + 2) * sizeof(float));
    if (tcw) b += align_up(4 * KC * KC * 2);
    if (sliced) b += align_up(resid_tc_slice_bytes((int)KC)) + align_up(2 * KC * sizeof(float));
    return b;
}
// Refining instances of the 128 and 256 classes whose residual runs with sliced
// products on the tensor cores (resid_tc.cu); the others keep the SIMT kernel.
// The slices' error, about 2^-28 of |A| |X|, reaches X through A^-1 twice, so
// channels with at most two antennas per user (Jacobi-scaled condition numbers
// up to thousands) keep the Dot2 residual.
bool sliced_resid(const jacpcg_config &cfg, bool refine, const jacpcg_instance &q) {
    return refine && cfg.refine_residual == JACPCG_RESID_SLICED && k_class(q.K) >= 128 && q.M > 2 * q.K;
}
constexpr int RTC_NB = 24;   // columns per job of the sliced residual

// K classes whose Gram runs on the tensor cores at this precision (64 x 64
// user-group blocks: one diagonal job for the 64 class, 2 + 1 for 128, 4 + 6
// for 256) ...
bool gram_on_tc(int precision, int KC) { return precision == JACPCG_TF32X3 && KC >= 64; }
// With refinement, channels with at most two antennas per user form A by the
// compensated SIMT Gram: their Jacobi-scaled condition numbers reach the
// thousands, and refinement converges to the solution for the A it is given,
// so the rounding of an FP32 (or 3xTF32) Gram would be the error floor of W.
bool accurate_gram(bool refine, const jacpcg_instance &q) { return refine && q.M <= 2 * q.K; }
// Instances that refinement works on: all of them, or with the selective
// policy only those with at most two antennas per user.
bool refines(const jacpcg_config &cfg, bool refine, const jacpcg_instance &q) {
    return refine && (!(cfg.flags & JACPCG_FLAG_REFINE_SELECTIVE) || q.M <= 2 * q.K);
}
// ... whose W = H X does (the 64 class with X resident, 128 and 256 with X
// streamed per stage, one job per 64 output columns) ...
bool hx_on_tc(int precision, int KC) { return precision == JACPCG_TF32X3 && KC >= 64; }
int hx_tc_groups(const jacpcg_instance &q) { return (n_cols(q) + 63) / 64; }
// ... and whose iteration does, unless the SIMT kernel is asked for (Algorithm 1
// and JOR always keep the SIMT kernel)
// (the K class's choice is -1: the tensor path where allowed)
bool tensor_iteration_allowed(const jacpcg_config &cfg, int KC) {
    return !(cfg.flags & JACPCG_FLAG_SIMT_ITERATION) && cfg.precision == JACPCG_TF32X3 && KC >= 64 &&
           (cfg.variant == JACPCG_STANDARD || cfg.variant == JACPCG_CG);
}
bool pcg_on_tc(const jacpcg_config &cfg, const int *shape_idx, int KC) {
    return KC == 64 && shape_idx[kc_index(KC)] < 0 && tensor_iteration_allowed(cfg, KC);
}
// ... and, for the 128 and 256 classes, the streamed-A tensor-core iteration
bool pcg_on_tcw(const jacpcg_config &cfg, const int *shape_idx, int KC) {
    return KC >= 128 && shape_idx[kc_index(KC)] < 0 && tensor_iteration_allowed(cfg, KC);
}

Layout make_layout(const jacpcg_config &cfg, const jacpcg_instance *inst, int n, bool refine,
                   const int *shape_idx) {
    Layout L{};
    L.n_gram = L.n_pcg = L.n_hx = L.n_res = L.n_gd = L.n_gx = L.n_hw = L.n_sinr = L.n_twj = 0;
    L.n_tm = L.n_gb = L.n_hb = L.n_rtl = L.n_rtj = 0;
    L.refine = refine;
    for (int i = 0; i < n; ++i) {
        if (refines(cfg, refine, inst[i])) {
            if (sliced_resid(cfg, refine, inst[i])) {
                ++L.n_rtl;
                L.n_rtj += (n_cols(inst[i]) + RTC_NB - 1) / RTC_NB;
            } else {
                L.n_res += (n_cols(inst[i]) + RES_CB - 1) / RES_CB;
            }
        }
        const int ng = k_class(inst[i].K) / 64;   // user groups of a tensor-core Gram
        L.n_gd += ng;
        L.n_gx += ng * (ng - 1) / 2;
        L.n_hw += hx_tc_groups(inst[i]);
        L.n_gram += n_gtiles(inst[i]);
        L.n_pcg += n_pblocks(inst[i], shape_idx);
        L.n_hx += n_wtiles(inst[i]);
        if (inst[i].sinr) L.n_sinr += (inst[i].K + 7) / 8;
        if (pcg_on_tcw(cfg, shape_idx, k_class(inst[i].K))) L.n_twj += (n_cols(inst[i]) + pcg_tcw_cols() - 1) / pcg_tcw_cols();
        if (bf16_native(cfg.precision, inst[i])) {
            L.n_tm += 2;   // the Gram's and W = H X's tensor maps
            if (!accurate_gram(refine, inst[i])) L.n_gb += k_class(inst[i].K) == 256 ? 3 : 1;
            L.n_hb += hx_bf16_groups(inst[i]);
        }
    }
    size_t o = 0;
    L.insts = o;  o += align_up(sizeof(DevInst) * n);
    L.gram = o;   o += align_up(sizeof(int4) * L.n_gram);
    L.tcl = o;    o += align_up(sizeof(int) * n);
    L.gdl = o;    o += align_up(sizeof(int2) * L.n_gd);
    L.gxl = o;    o += align_up(sizeof(int4) * L.n_gx);
    L.pcg = o;    o += align_up(sizeof(int2) * L.n_pcg);
    L.hx = o;     o += align_up(sizeof(int4) * L.n_hx);
    L.hxl = o;    o += align_up(sizeof(int) * n);
    L.hwl = o;    o += align_up(sizeof(int2) * L.n_hw);
    L.res = o;    o += align_up(sizeof(int2) * L.n_res);
    L.rtl = o;    o += align_up(sizeof(int) * L.n_rtl);
    L.rtj = o;    o += align_up(sizeof(int2) * L.n_rtj);
    L.sinr = o;   o += align_up(sizeof(int2) * L.n_sinr);
    L.twl = o;    o += align_up(sizeof(int) * n);
    L.twj = o;    o += align_up(sizeof(int2) * L.n_twj);
    L.tmaps = o;  o += align_up(sizeof(CUtensorMap) * L.n_tm);
    L.gbl = o;    o += align_up(sizeof(int4) * L.n_gb);
    L.hbl = o;    o += align_up(sizeof(int4) * L.n_hb);
    L.accum = o;  o += align_up(sizeof(int32_t) * n) * 3;
    L.ws = o;
    L.ws_off.resize(n);
    for (int i = 0; i < n; ++i) {
        L.ws_off[i] = o;
        o += inst_ws_bytes(inst[i], refine, pcg_on_tcw(cfg, shape_idx, k_class(inst[i].K)),
                           refines(cfg, refine, inst[i]) && sliced_resid(cfg, refine, inst[i]));
    }
    L.total = o;
    return L;
}

// Fill the host image of the table part ([0, L.accum)) for a block at `dev`
// and the launch list of the plan.
// Tensor maps over a bfloat16 channel's H read as K rows of 2M values (row
// stride ldh * 4 bytes), 128-byte swizzle, zero fill past M and K: box 64 x 128
// (64 values of 128 users) for the Gram's user tiles and W = H X's stages.
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
bool encode_h_maps(const jacpcg_ctx *ctx, const jacpcg_instance &q, CUtensorMap *gram_map, CUtensorMap *hx_map) {
    if (!ctx->encode) return false;
    const EncodeTiled enc = reinterpret_cast<EncodeTiled>(ctx->encode);
    const cuuint64_t dims[2] = {2 * (cuuint64_t)q.M, (cuuint64_t)q.K};
    const cuuint64_t strides[1] = {4 * (cuuint64_t)q.ldh};
    const cuuint32_t elem[2] = {1, 1};
    const cuuint32_t gbox[2] = {64, 128}, hbox[2] = {64, 128};   // the same box: 64 values x 128 users
    void *base = const_cast<void *>(q.H);
    return enc(gram_map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, gbox, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
           enc(hx_map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, hbox, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool build_tables(const jacpcg_ctx *ctx, const jacpcg_instance *inst, int n, const Layout &L,
                  char *dev, char *host, std::vector<Launch> &launches) {
    DevInst *hi = reinterpret_cast<DevInst *>(host + L.insts);
    for (int i = 0; i < n; ++i) {
        const jacpcg_instance &q = inst[i];
        const int KC = k_class(q.K);
        char *w = dev + L.ws_off[i];
        DevInst d{};
        d.H = static_cast<const float2 *>(q.H);
        d.W = static_cast<float2 *>(q.W);
        d.Xout = static_cast<float2 *>(q.X);
        d.Aout = static_cast<float2 *>(q.A);
        d.A = reinterpret_cast<float2 *>(w);
        d.X = reinterpret_cast<float2 *>(w + align_up((size_t)KC * KC * sizeof(float2)));
        d.dinv = reinterpret_cast<float *>(w + 2 * align_up((size_t)KC * KC * sizeof(float2)));
        d.wpart = reinterpret_cast<float *>(w + 2 * align_up((size_t)KC * KC * sizeof(float2)) +
                                            align_up(KC * sizeof(float)));
        d.M = q.M; d.K = q.K; d.ldh = q.ldh; d.ldw = q.ldw; d.KC = KC;
        d.max_iter = q.max_iter;
        d.n_wpart = !hx_on_tc(ctx->cfg.precision, KC)   ? n_wtiles(q)
                    : bf16_native(ctx->cfg.precision, q) ? hx_bf16_slots(q)
                    : KC == 64                           ? (q.M + 127) / 128
                                                         : ((q.M + 127) / 128) * hx_tc_groups(q);
        d.variant = ctx->cfg.variant;
        d.omega = q.omega > 0.f ? q.omega : 1.f;
        d.sinr = q.sinr;
        d.noise = q.noise;
        d.xi = (float)q.xi;
        d.power = q.power > 0.0 ? (float)q.power : 1.0f;
        d.tol = q.tol;
        d.h_bf16 = q.h_dtype == JACPCG_H_BF16;
        d.B = static_cast<const float2 *>(q.B);
        d.ldb = q.B ? q.ldb : 0;
        d.ncols = n_cols(q);
        d.X0 = static_cast<const float2 *>(q.X0);
        const bool tcw_i = pcg_on_tcw(ctx->cfg, ctx->pcg_shape_idx, KC);
        if (tcw_i) {   // the split stages follow everything else
            d.As = reinterpret_cast<float *>(w + inst_ws_bytes(q, L.refine, false));
        }
        if (refines(ctx->cfg, L.refine, q) && sliced_resid(ctx->cfg, L.refine, q)) {   // then A's slices
            const size_t o = inst_ws_bytes(q, L.refine, tcw_i);
            d.Asl = w + o;
            d.rexp = reinterpret_cast<float *>(w + o + align_up(resid_tc_slice_bytes(KC)));
        }
        if (L.refine) {
            const size_t base = 2 * align_up((size_t)KC * KC * sizeof(float2)) + align_up(KC * sizeof(float)) +
                                align_up(wpart_slots(q) * sizeof(float));
            d.R = reinterpret_cast<float2 *>(w + base);
            d.rnorm = reinterpret_cast<float *>(w + base + align_up((size_t)KC * KC * sizeof(float2)));
            d.rctl = d.rnorm + 2 * KC;
            d.rtol2 = ctx->cfg.refine_tol * ctx->cfg.refine_tol;
            d.no_refine = refines(ctx->cfg, true, q) ? 0 : 1;
            d.rsolve_tol = ctx->cfg.refine_solve_tol;
            d.resid_hist = q.resid_hist;
        }
        hi[i] = d;
    }
    launches.clear();
    if (L.refine) {   // residual blocks: (instance, column); the sliced residual's lists per K class
        int2 *rb = reinterpret_cast<int2 *>(host + L.res);
        int r = 0;
        for (int i = 0; i < n; ++i)
            if (refines(ctx->cfg, true, inst[i]) && !sliced_resid(ctx->cfg, true, inst[i]))
                for (int j = 0; j < n_cols(inst[i]); j += RES_CB) rb[r++] = make_int2(i, j);
        int *rl = reinterpret_cast<int *>(host + L.rtl);
        int2 *rj = reinterpret_cast<int2 *>(host + L.rtj);
        int nl = 0, nj = 0;
        for (int KC : {128, 256}) {
            const int l0 = nl, j0 = nj;
            for (int i = 0; i < n; ++i) {
                if (k_class(inst[i].K) != KC || !refines(ctx->cfg, true, inst[i]) ||
                    !sliced_resid(ctx->cfg, true, inst[i]))
                    continue;
                rl[nl++] = i;
                for (int c0 = 0; c0 < n_cols(inst[i]); c0 += RTC_NB) rj[nj++] = make_int2(i, c0);
            }
            if (nl > l0)
                launches.push_back({Launch::RESID_TC, 4, KC, L.rtl + l0 * sizeof(int), nl - l0, 0,
                                    L.rtj + j0 * sizeof(int2), nj - j0});
        }
    }
    // Gram on the tensor cores: diagonal (instance, group) jobs, then the
    // off-diagonal (instance, a, b) jobs of the 128 and 256 classes
    const int prec = ctx->cfg.precision;
    int2 *gd = reinterpret_cast<int2 *>(host + L.gdl);
    int4 *gx = reinterpret_cast<int4 *>(host + L.gxl);
    int nd = 0, nx = 0;
    for (int i = 0; i < n; ++i) {
        const int KC = k_class(inst[i].K);
        if (!gram_on_tc(prec, KC) || accurate_gram(L.refine, inst[i]) || bf16_native(prec, inst[i])) continue;
        for (int a = 0; a < KC / 64; ++a) {
            gd[nd++] = make_int2(i, a);
            for (int b = a + 1; b < KC / 64; ++b) gx[nx++] = make_int4(i, a, b, 0);
        }
    }
    if (nd) launches.push_back({Launch::GRAM_TC, 0, 0, L.gdl, nd});
    if (nx) launches.push_back({Launch::GRAM_TCX, 0, 0, L.gxl, nx});
    // bfloat16 channels of the 128 and 256 classes: two tensor maps each, the
    // Gram's (instance, tile a, tile b >= a) jobs and W = H X's (instance, group) jobs
    CUtensorMap *tm = reinterpret_cast<CUtensorMap *>(host + L.tmaps);
    int4 *gb = reinterpret_cast<int4 *>(host + L.gbl);
    int4 *hb = reinterpret_cast<int4 *>(host + L.hbl);
    int nm = 0, ngb = 0, nhb = 0;
    for (int i = 0; i < n; ++i) {
        if (!bf16_native(prec, inst[i])) continue;
        if (!encode_h_maps(ctx, inst[i], tm + nm, tm + nm + 1)) return false;
        const int nt = k_class(inst[i].K) / 128;
        if (!accurate_gram(L.refine, inst[i]))
            for (int a = 0; a < nt; ++a)
                for (int b = a; b < nt; ++b) gb[ngb++] = make_int4(i, a, b, nm);
        for (int g = 0; g < hx_bf16_groups(inst[i]); ++g) hb[nhb++] = make_int4(i, g, nm + 1, 0);
        nm += 2;
    }
    if (ngb) launches.push_back({Launch::GRAM_BF16, 0, 0, L.gbl, ngb});
    // the K = 64 class's tensor-core iteration: instance list
    int *tl = reinterpret_cast<int *>(host + L.tcl);
    int nt = 0;
    for (int i = 0; i < n; ++i)
        if (pcg_on_tc(ctx->cfg, ctx->pcg_shape_idx, k_class(inst[i].K))) tl[nt++] = i;
    // Gram tiles (SIMT) grouped by tile edge
    int4 *gt = reinterpret_cast<int4 *>(host + L.gram);
    int g = 0;
    for (int accurate = 0; accurate < 2; ++accurate) {
        for (int TB : {16, 32, 64}) {
            const int start = g;
            for (int i = 0; i < n; ++i) {
                const int KC = k_class(inst[i].K);
                const bool acc_i = accurate_gram(L.refine, inst[i]);
                if (gram_tb(KC) != TB || acc_i != (accurate != 0) || (!acc_i && gram_on_tc(prec, KC))) continue;
                const int nb = std::max(1, KC / TB);
                for (int bi = 0; bi < nb; ++bi)
                    for (int bj = 0; bj <= bi; ++bj) gt[g++] = make_int4(i, bi, bj, 0);
            }
            // Launch::shape carries the compensated flag of a SIMT Gram launch
            if (g > start) launches.push_back({Launch::GRAM, 0, TB, L.gram + start * sizeof(int4), g - start, accurate});
        }
    }
    // iteration blocks grouped by K class
    int2 *pb = reinterpret_cast<int2 *>(host + L.pcg);
    int p = 0;
    if (nt) launches.push_back({Launch::PCG_TC, 1, 64, L.tcl, nt});
    // the 128 and 256 classes on the tensor cores: split A once, then the jobs
    // (instance, 32 columns), instance-major so that the CTAs of an instance
    // stream its A from L2 at about the same time
    {
        int *twl = reinterpret_cast<int *>(host + L.twl);
        int2 *twj = reinterpret_cast<int2 *>(host + L.twj);
        int ni = 0, nj = 0;
        for (int KC : {128, 256}) {
            if (!pcg_on_tcw(ctx->cfg, ctx->pcg_shape_idx, KC)) continue;
            const int i0 = ni, j0 = nj;
            for (int i = 0; i < n; ++i) {
                if (k_class(inst[i].K) != KC) continue;
                twl[ni++] = i;
                for (int c0 = 0; c0 < n_cols(inst[i]); c0 += pcg_tcw_cols()) twj[nj++] = make_int2(i, c0);
            }
            if (ni > i0) {
                launches.push_back({Launch::TCW_PREP, 1, KC, L.twl + i0 * sizeof(int), ni - i0});
                launches.push_back({Launch::PCG_TCW, 1, KC, L.twj + j0 * sizeof(int2), nj - j0});
            }
        }
    }
    if (ctx->cfg.variant == JACPCG_DIRECT) {   // direct solve: instance lists per K class
        int c = 0;
        for (int KC : {8, 16, 32, 64, 128, 256}) {
            const int start = c;
            for (int i = 0; i < n; ++i)
                if (k_class(inst[i].K) == KC) tl[c++] = i;
            if (c > start) launches.push_back({Launch::CHOL, 1, KC, L.tcl + start * sizeof(int), c - start});
        }
    }
    for (int KC : {8, 16, 32, 64, 128, 256}) {
        if (ctx->cfg.variant == JACPCG_DIRECT) break;
        const int start = p;
        const int sh = ctx->pcg_shape_idx[kc_index(KC)] < 0 ? 0 : ctx->pcg_shape_idx[kc_index(KC)];
        const PcgShape s = pcg_shape(KC, sh);
        for (int i = 0; i < n; ++i) {
            if (k_class(inst[i].K) != KC || pcg_on_tc(ctx->cfg, ctx->pcg_shape_idx, KC) ||
                pcg_on_tcw(ctx->cfg, ctx->pcg_shape_idx, KC))
                continue;
            for (int c0 = 0; c0 < n_cols(inst[i]); c0 += s.CW * s.NW) pb[p++] = make_int2(i, c0);
        }
        if (p > start) launches.push_back({Launch::PCG, 1, KC, L.pcg + start * sizeof(int2), p - start, sh});
    }
    // W = H X on the tensor cores: instance list, one persistent launch
    int *hl = reinterpret_cast<int *>(host + L.hxl);
    int nh = 0;
    for (int i = 0; i < n; ++i)
        if (hx_on_tc(prec, k_class(inst[i].K)) && k_class(inst[i].K) == 64) hl[nh++] = i;
    if (nh) launches.push_back({Launch::HX_TC, 2, 0, L.hxl, nh});
    int2 *hw = reinterpret_cast<int2 *>(host + L.hwl);
    int nw = 0;
    for (int i = 0; i < n; ++i)
        if (hx_on_tc(prec, k_class(inst[i].K)) && k_class(inst[i].K) > 64 && !bf16_native(prec, inst[i]))
            for (int b = 0; b < hx_tc_groups(inst[i]); ++b) hw[nw++] = make_int2(i, b);
    if (nw) launches.push_back({Launch::HX_TCW, 2, 0, L.hwl, nw});
    if (nhb) launches.push_back({Launch::HX_BF16, 2, 0, L.hbl, nhb});
    // W = H X tiles (SIMT) grouped by tile width; slot = index of the tile in its instance
    int4 *ht = reinterpret_cast<int4 *>(host + L.hx);
    int h = 0;
    for (int TN : {16, 32, 64}) {
        const int start = h;
        for (int i = 0; i < n; ++i) {
            const int KC = k_class(inst[i].K);
            if (hx_tn(KC) != TN || hx_on_tc(prec, KC)) continue;
            const int nm = (inst[i].M + HX_TM - 1) / HX_TM, nn = (n_cols(inst[i]) + TN - 1) / TN;
            int slot = 0;
            for (int nt = 0; nt < nn; ++nt)
                for (int mt = 0; mt < nm; ++mt) ht[h++] = make_int4(i, mt, nt, slot++);
        }
        if (h > start) launches.push_back({Launch::HX, 2, TN, L.hx + start * sizeof(int4), h - start});
    }
    // per-user SINR (Eq. 9) after the power factor: (instance, block of 8 users) jobs per K class
    int2 *sj = reinterpret_cast<int2 *>(host + L.sinr);
    int ns = 0;
    for (int KC : {8, 16, 32, 64, 128, 256}) {
        const int start = ns;
        for (int i = 0; i < n; ++i)
            if (inst[i].sinr && k_class(inst[i].K) == KC)
                for (int b = 0; b < (inst[i].K + 7) / 8; ++b) sj[ns++] = make_int2(i, b);
        if (ns > start) launches.push_back({Launch::SINR, 3, KC, L.sinr + start * sizeof(int2), ns - start});
    }
    return true;
}

constexpr size_t MAX_PROFILED = 4096;

// NVTX range around the host-side enqueue of one phase: Nsight tools show the
// phases by name and attribute their kernels; without a tool attached each
// push / pop is a no-op.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

jacpcg_status enqueue(jacpcg_plan *pl, cudaStream_t s, bool profile, int *n_launched) {
    jacpcg_ctx *ctx = pl->ctx;
    int nl = 0;
    cudaEvent_t *ev = nullptr;
    if (profile && ctx->prof_used < MAX_PROFILED) {
        if (ctx->prof_used == ctx->prof_pool.size()) {
            std::array<cudaEvent_t, 5> set{};
            for (auto &e : set) CK(cudaEventCreate(&e));
            ctx->prof_pool.push_back(set);
        }
        ev = ctx->prof_pool[ctx->prof_used++].data();
    }
    if (ev) CK(cudaEventRecord(ev[0], s));
    if (pl->acc_reset_bytes) {   // several Gram jobs per instance report into shared accumulators
        CK(cudaMemsetAsync(pl->acc.flags, 0, pl->acc_reset_bytes, s));
    }
    static const char *const kPhase[3] = {"jacpcg: Gram", "jacpcg: iteration", "jacpcg: W = H X"};
    for (int phase = 0; phase < 3; ++phase) {
        const NvtxRange range(kPhase[phase]);
        for (const Launch &l : pl->launches) {
            if (l.phase != phase) continue;
            cudaError_t e = cudaSuccess;
            const void *list = pl->dev + l.list_off;
            switch (l.kind) {
                case Launch::GRAM:
                    e = launch_gram_simt(l.param, pl->d_insts, static_cast<const int4 *>(list), l.count,
                                         pl->acc, s, l.shape != 0);
                    break;
                case Launch::PCG:
                    e = launch_pcg_shape(l.param, l.shape, ctx->cfg.variant, pl->d_insts,
                                         static_cast<const int2 *>(list), l.count, pl->acc, s, 0);
                    break;
                case Launch::HX:
                    e = launch_hx_simt(l.param, pl->d_insts, static_cast<const int4 *>(list), l.count,
                                       s);
                    break;
                case Launch::GRAM_TC:
                    e = launch_gram_tc64(pl->d_insts, static_cast<const int2 *>(list), l.count, pl->acc, s);
                    break;
                case Launch::GRAM_TCX:
                    e = launch_gram_tc_cross(pl->d_insts, static_cast<const int4 *>(list), l.count, pl->acc, s);
                    break;
                case Launch::HX_TC:
                    e = launch_hx_tc64(pl->d_insts, static_cast<const int *>(list), l.count, pl->acc, s);
                    break;
                case Launch::HX_TCW:
                    e = launch_hx_tc_wide(pl->d_insts, static_cast<const int2 *>(list), l.count, pl->acc, s);
                    break;
                case Launch::PCG_TC:
                    e = launch_pcg_tc64(ctx->cfg.variant, pl->d_insts, static_cast<const int *>(list), l.count,
                                        pl->acc, &ctx->amap, ctx->arena.base, s, 0);
                    break;
                case Launch::CHOL:
                    e = launch_chol(l.param, pl->d_insts, static_cast<const int *>(list), l.count, pl->acc, s);
                    break;
                case Launch::TCW_PREP:
                    e = launch_tcw_prep(l.param, pl->d_insts, static_cast<const int *>(list), l.count, s);
                    break;
                case Launch::PCG_TCW:
                    e = launch_pcg_tcw(l.param, ctx->cfg.variant, pl->d_insts, static_cast<const int2 *>(list),
                                       l.count, pl->acc, s, 0);
                    break;
                case Launch::GRAM_BF16:
                    e = launch_gram_bf16(pl->d_insts, static_cast<const int4 *>(list), l.count,
                                         reinterpret_cast<const CUtensorMap *>(pl->dev + pl->tmap_off), pl->acc, s);
                    break;
                case Launch::HX_BF16:
                    e = launch_hx_bf16(pl->d_insts, static_cast<const int4 *>(list), l.count,
                                       reinterpret_cast<const CUtensorMap *>(pl->dev + pl->tmap_off), pl->acc, s);
                    break;
                case Launch::RESID_TC:   // phase 4: run by the refinement below
                    break;
            }
            if (e != cudaSuccess) return cuda_fail(ctx, e);
            ++nl;
        }
        if (phase == 1 && pl->refine_sweeps > 0 && (pl->n_res > 0 || pl->n_rtc > 0)) {   // some instance refines
            // iterative refinement: R = I - A X (Dot2, FP64 or sliced), A dX = R (FP32 iteration), X += dX
            const NvtxRange refine_range("jacpcg: refinement");
            const int2 *rb = reinterpret_cast<const int2 *>(pl->dev + pl->res_off);
            for (const Launch &l : pl->launches) {   // A's slices, once per execute
                if (l.kind != Launch::RESID_TC) continue;
                if (launch_rtc_prep(l.param, pl->d_insts, reinterpret_cast<const int *>(pl->dev + l.list_off), l.count,
                                    s) != cudaSuccess)
                    return cuda_fail(ctx);
                ++nl;
            }
            for (int sw = 0; sw <= pl->refine_sweeps; ++sw) {
                // after the last correction the residual could only be reported
                if (sw == pl->refine_sweeps && !pl->want_hist) break;
                if (pl->n_res > 0) {
                    if (launch_residual(pl->d_insts, rb, pl->n_res, sw, s,
                                        ctx->cfg.refine_residual == JACPCG_RESID_FP64) != cudaSuccess)
                        return cuda_fail(ctx);
                    ++nl;
                }
                for (const Launch &l : pl->launches) {
                    if (l.kind != Launch::RESID_TC) continue;
                    if (launch_resid_tc(l.param, pl->d_insts, reinterpret_cast<const int2 *>(pl->dev + l.list2_off),
                                        l.count2, sw, pl->acc, s) != cudaSuccess)
                        return cuda_fail(ctx);
                    ++nl;
                }
                if (launch_resid_hist(pl->d_insts, pl->n_inst, sw, s) != cudaSuccess) return cuda_fail(ctx);
                ++nl;
                if (sw == pl->refine_sweeps) break;
                for (const Launch &l : pl->launches) {
                    cudaError_t e = cudaSuccess;
                    if (l.kind == Launch::PCG)
                        e = launch_pcg_shape(l.param, l.shape, ctx->cfg.variant, pl->d_insts,
                                             reinterpret_cast<const int2 *>(pl->dev + l.list_off), l.count,
                                             pl->acc, s, 1);
                    else if (l.kind == Launch::PCG_TC)
                        e = launch_pcg_tc64(ctx->cfg.variant, pl->d_insts,
                                            reinterpret_cast<const int *>(pl->dev + l.list_off), l.count,
                                            pl->acc, &ctx->amap, ctx->arena.base, s, 1);
                    else if (l.kind == Launch::PCG_TCW)   // loose corrections: heads only (mode 2)
                        e = launch_pcg_tcw(l.param, ctx->cfg.variant, pl->d_insts,
                                           reinterpret_cast<const int2 *>(pl->dev + l.list_off), l.count,
                                           pl->acc, s, ctx->cfg.refine_solve_tol >= 5e-3f ? 2 : 1);
                    else
                        continue;
                    if (e != cudaSuccess) return cuda_fail(ctx, e);
                    ++nl;
                }
            }
        }
        if (ev) CK(cudaEventRecord(ev[phase + 1], s));
    }
    {
        const NvtxRange range("jacpcg: finalize");
        const cudaError_t e = launch_finalize(pl->d_insts, pl->n_inst, pl->acc, pl->out, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
    }
    ++nl;
    for (const Launch &l : pl->launches) {
        if (l.phase != 3) continue;
        const NvtxRange range("jacpcg: SINR");
        const cudaError_t e = launch_sinr(l.param, pl->d_insts, reinterpret_cast<const int2 *>(pl->dev + l.list_off),
                                          l.count, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
        ++nl;
    }
    if (ev) CK(cudaEventRecord(ev[4], s));
    *n_launched = nl;
    return JACPCG_OK;
}

jacpcg_status make_plan(jacpcg_ctx *ctx, const jacpcg_instance *inst, int n, int32_t *status_dev,
                        int32_t *iters_dev, float *resid_dev, float *beta_dev, int use_graph,
                        cudaStream_t async_stream, jacpcg_plan **out) {
    if (!ctx || !out) return JACPCG_EINVAL;
    if (ctx->broken) return JACPCG_ECUDA;
    jacpcg_status st = validate(ctx, inst, n);
    if (st != JACPCG_OK) return st;
    const bool refine = ctx->cfg.refine_sweeps > 0;
    Layout L = make_layout(ctx->cfg, inst, n, refine, ctx->pcg_shape_idx);
    size_t off;
    if (!ctx->arena.alloc(L.total, &off)) return JACPCG_ENOMEM;
    jacpcg_plan *pl = new (std::nothrow) jacpcg_plan();
    if (!pl) {
        ctx->arena.release(off, L.total, nullptr);
        return JACPCG_ENOMEM;
    }
    pl->ctx = ctx;
    pl->off = off;
    pl->bytes = L.total;
    pl->dev = ctx->arena.base + off;
    pl->n_inst = n;
    pl->d_insts = reinterpret_cast<DevInst *>(pl->dev + L.insts);
    pl->acc.flags = reinterpret_cast<int32_t *>(pl->dev + L.accum);
    pl->acc.iters = reinterpret_cast<int32_t *>(pl->dev + L.accum + align_up(sizeof(int32_t) * n));
    pl->acc.resid_bits =
        reinterpret_cast<uint32_t *>(pl->dev + L.accum + 2 * align_up(sizeof(int32_t) * n));
    pl->out = DevOut{status_dev, iters_dev, resid_dev, beta_dev};
    pl->use_graph = use_graph;
    pl->refine_sweeps = ctx->cfg.refine_sweeps;
    for (int i = 0; i < n; ++i) pl->want_hist = pl->want_hist || inst[i].resid_hist != nullptr;
    pl->res_off = L.res;
    pl->n_res = L.n_res;
    pl->n_rtc = L.n_rtl;
    if (L.n_gx || L.n_gb) pl->acc_reset_bytes = 3 * align_up(sizeof(int32_t) * n);
    pl->tmap_off = L.tmaps;
    const size_t tbytes = L.accum;   // tables occupy [0, accum)
    auto fail = [&](jacpcg_status s) {
        ctx->arena.release(pl->off, pl->bytes, nullptr);
        delete pl;
        return s;
    };
    // host image in pinned staging, uploaded on the stream (or synchronously)
    if (ctx->staging_pending) {
        if (cudaEventSynchronize(ctx->staging_ev) != cudaSuccess) return fail(cuda_fail(ctx));
        ctx->staging_pending = false;
    }
    if (ctx->staging_bytes < tbytes) {
        if (ctx->staging) cudaFreeHost(ctx->staging);
        ctx->staging = nullptr;
        ctx->staging_bytes = 0;
        if (cudaHostAlloc(reinterpret_cast<void **>(&ctx->staging), tbytes, cudaHostAllocDefault) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            return fail(JACPCG_ENOMEM);
        }
        ctx->staging_bytes = tbytes;
    }
    std::memset(ctx->staging, 0, tbytes);
    if (!build_tables(ctx, inst, n, L, pl->dev, ctx->staging, pl->launches)) return fail(JACPCG_ECUDA);
    if (async_stream) {
        if (cudaMemcpyAsync(pl->dev, ctx->staging, tbytes, cudaMemcpyHostToDevice, async_stream) !=
                cudaSuccess ||
            cudaEventRecord(ctx->staging_ev, async_stream) != cudaSuccess)
            return fail(cuda_fail(ctx));
        ctx->staging_pending = true;
    } else {
        if (cudaMemcpy(pl->dev, ctx->staging, tbytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(cuda_fail(ctx));
    }
    if (cudaEventCreateWithFlags(&pl->done, cudaEventDisableTiming) != cudaSuccess)
        return fail(cuda_fail(ctx));
    ctx->plans.push_back(pl);
    *out = pl;
    return JACPCG_OK;
}

void drop_plan(jacpcg_plan *pl) {
    jacpcg_ctx *ctx = pl->ctx;
    if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
    // the block is reused only after the plan's last execute has finished
    ctx->arena.release(pl->off, pl->bytes, pl->executed ? pl->done : nullptr);
    if (!pl->executed && pl->done) cudaEventDestroy(pl->done);
    ctx->plans.erase(std::remove(ctx->plans.begin(), ctx->plans.end(), pl), ctx->plans.end());
    delete pl;
}

jacpcg_status execute(jacpcg_plan *pl, cudaStream_t s) {
    jacpcg_ctx *ctx = pl->ctx;
    if (ctx->broken) return JACPCG_ECUDA;
    const bool profile = (ctx->cfg.flags & JACPCG_FLAG_PROFILE) && !pl->use_graph;
    int nl = 0;
    if (pl->use_graph) {
        if (!pl->gexec) {
            // capture on the context's own stream (the caller's may be the
            // legacy default stream, which cannot be captured)
            cudaGraph_t g = nullptr;
            const cudaStream_t cs = ctx->capture_stream;
            CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            jacpcg_status st = enqueue(pl, cs, false, &pl->graph_launches);
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (st != JACPCG_OK) return st;
            if (e != cudaSuccess) return cuda_fail(ctx);
            e = cudaGraphInstantiate(&pl->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(ctx);
        }
        CK(cudaGraphLaunch(pl->gexec, s));
        nl = pl->graph_launches;
    } else {
        jacpcg_status st = enqueue(pl, s, profile, &nl);
        if (st != JACPCG_OK) return st;
    }
    ctx->last_launches = nl;
    ctx->launches += nl;
    CK(cudaEventRecord(pl->done, s));
    pl->executed = true;
    return JACPCG_OK;
}

// The arena as a 2-D FP32 tensor: one row of 64 floats per 256-byte allocation
// unit, so every workspace block (A of a K = 64 instance: 128 rows) starts at a
// row.  The tensor-core iteration stages A with one tiled TMA copy of a 64 x 128
// box.  The encoder is the driver's, reached through the runtime.
bool encode_arena_map(jacpcg_ctx *ctx) {
    static_assert(ALIGN == 256, "arena rows are 256 bytes");
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        (void)cudaGetLastError();
        return false;
    }
    const cuuint64_t dims[2] = {64, ctx->arena.size / ALIGN};
    const cuuint64_t strides[1] = {ALIGN};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t elem[2] = {1, 1};
    ctx->encode = fn;
    return reinterpret_cast<Encode>(fn)(&ctx->amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ctx->arena.base, dims,
                                        strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

const char *jacpcg_version(void) { return "0.1.0"; }

// Eq. 7: each block of the block precoder is an RZF of its own sub-channel;
// the sub-instances point into the full channel and the full W.
jacpcg_status jacpcg_blocks(const jacpcg_instance *full, const jacpcg_block *blocks, int n_blocks,
                            jacpcg_instance *out) {
    if (!full || !blocks || !out || n_blocks < 1 || !full->H || !full->W) return JACPCG_EINVAL;
    const size_t hes = full->h_dtype == JACPCG_H_BF16 ? 4 : 8;
    for (int b = 0; b < n_blocks; ++b) {
        const jacpcg_block &k = blocks[b];
        if (k.rows < 1 || k.cols < 1 || k.row0 < 0 || k.col0 < 0 || k.row0 + k.rows > full->M ||
            k.col0 + k.cols > full->K)
            return JACPCG_EINVAL;
        if (k.cols > k.rows && !(full->xi > 0.0)) return JACPCG_EINVAL;
        const size_t ho = ((size_t)k.col0 * full->ldh + k.row0) * hes;
        const size_t wo = ((size_t)k.col0 * full->ldw + k.row0) * 8;
        if (!aligned16(static_cast<const char *>(full->H) + ho) ||
            !aligned16(static_cast<const char *>(full->W) + wo))
            return JACPCG_EINVAL;
    }
    for (int b = 0; b < n_blocks; ++b) {
        const jacpcg_block &k = blocks[b];
        jacpcg_instance q = *full;
        q.M = k.rows;
        q.K = k.cols;
        q.H = static_cast<const char *>(full->H) + ((size_t)k.col0 * full->ldh + k.row0) * hes;
        q.W = static_cast<char *>(full->W) + ((size_t)k.col0 * full->ldw + k.row0) * 8;
        q.X = nullptr;
        q.A = nullptr;
        q.resid_hist = nullptr;
        q.B = nullptr;
        q.ldb = 0;
        q.n_rhs = 0;
        q.X0 = nullptr;
        out[b] = q;
    }
    return JACPCG_OK;
}

const char *jacpcg_strerror(jacpcg_status s) {
    switch (s) {
        case JACPCG_OK: return "ok";
        case JACPCG_EINVAL: return "invalid argument";
        case JACPCG_ENOMEM: return "out of memory (device, pinned host or arena budget)";
        case JACPCG_ECUDA: return "CUDA runtime error; context unusable";
        case JACPCG_ENOTCONV: return "tolerance not met within max_iter";
        case JACPCG_ENOTHPD: return "matrix not Hermitian positive definite";
        case JACPCG_ENONFINITE: return "non-finite value in the precoder";
        case JACPCG_ETIMEOUT: return "bounded wait ran out";
        case JACPCG_EBUSY: return "busy";
    }
    return "unknown status";
}

jacpcg_status jacpcg_create(const jacpcg_config *cfg, jacpcg_ctx **out) {
    if (!cfg || !out) return JACPCG_EINVAL;
    if (cfg->max_K < 1 || cfg->max_K > 256 || cfg->max_M < 1 || cfg->max_instances < 1)
        return JACPCG_EINVAL;
    if (cfg->precision != JACPCG_FP32 && cfg->precision != JACPCG_TF32X3) return JACPCG_EINVAL;
    if (cfg->variant < JACPCG_STANDARD || cfg->variant > JACPCG_DIRECT) return JACPCG_EINVAL;
    if (cfg->variant == JACPCG_DIRECT && cfg->refine_sweeps > 0) return JACPCG_EINVAL;
    if (cfg->flags & ~(JACPCG_FLAG_PROFILE | JACPCG_FLAG_SIMT_ITERATION | JACPCG_FLAG_REFINE_SELECTIVE))
        return JACPCG_EINVAL;
    if (cfg->refine_sweeps < 0 || cfg->refine_sweeps > 3) return JACPCG_EINVAL;
    if (cfg->refine_residual != JACPCG_RESID_DOT2 && cfg->refine_residual != JACPCG_RESID_FP64 &&
        cfg->refine_residual != JACPCG_RESID_SLICED)
        return JACPCG_EINVAL;
    if (!(cfg->refine_tol >= 0.f) || cfg->refine_tol > 1e30f) return JACPCG_EINVAL;   // also NaN
    if (!(cfg->refine_solve_tol >= 0.f) || cfg->refine_solve_tol > 1e30f) return JACPCG_EINVAL;
    jacpcg_ctx *ctx = new (std::nothrow) jacpcg_ctx();
    if (!ctx) return JACPCG_ENOMEM;
    ctx->cfg = *cfg;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete ctx;
        return JACPCG_EINVAL;
    }
    size_t bytes = cfg->arena_bytes;
    if (bytes == 0) {
        jacpcg_instance q{};
        q.M = cfg->max_M;
        q.K = cfg->max_K;
        std::vector<jacpcg_instance> v(cfg->max_instances, q);
        const int dflt[6] = {-1, -1, -1, -1, -1, -1};
        bytes = 2 * make_layout(*cfg, v.data(), cfg->max_instances, cfg->refine_sweeps > 0, dflt).total;
    }
    bytes = align_up(bytes);
    if (cudaMalloc(reinterpret_cast<void **>(&ctx->arena.base), bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        delete ctx;
        return JACPCG_ENOMEM;
    }
    ctx->arena.size = bytes;
    ctx->arena.free_.emplace(0, bytes);
    bool ok = cudaEventCreateWithFlags(&ctx->staging_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) == cudaSuccess &&
              encode_arena_map(ctx);
    if (!ok) {
        (void)cudaGetLastError();
        jacpcg_destroy(ctx);
        return JACPCG_ECUDA;
    }
    *out = ctx;
    return JACPCG_OK;
}

jacpcg_status jacpcg_destroy(jacpcg_ctx *ctx) {
    if (!ctx) return JACPCG_EINVAL;
    cudaSetDevice(ctx->cfg.device);
    cudaDeviceSynchronize();
    while (!ctx->plans.empty()) drop_plan(ctx->plans.back());
    ctx->arena.reap(false);
    for (auto &p : ctx->arena.pending) cudaEventDestroy(p.ev);
    if (ctx->arena.base) cudaFree(ctx->arena.base);
    if (ctx->staging) cudaFreeHost(ctx->staging);
    if (ctx->staging_ev) cudaEventDestroy(ctx->staging_ev);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    for (auto &set : ctx->prof_pool)
        for (auto &e : set) cudaEventDestroy(e);
    (void)cudaGetLastError();
    delete ctx;
    return JACPCG_OK;
}

jacpcg_status jacpcg_plan_create(jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst,
                                 int32_t *status_dev, int32_t *iters_dev, float *resid_dev,
                                 float *beta_dev, int use_graph, jacpcg_plan **out) {
    return make_plan(ctx, inst, n_inst, status_dev, iters_dev, resid_dev, beta_dev, use_graph,
                     nullptr, out);
}

jacpcg_status jacpcg_plan_execute(jacpcg_plan *plan, void *stream) {
    if (!plan) return JACPCG_EINVAL;
    return execute(plan, static_cast<cudaStream_t>(stream));
}

jacpcg_status jacpcg_plan_destroy(jacpcg_plan *plan) {
    if (!plan) return JACPCG_EINVAL;
    drop_plan(plan);
    return JACPCG_OK;
}

jacpcg_status jacpcg_precode(jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst,
                             int32_t *status_dev, int32_t *iters_dev, float *resid_dev,
                             float *beta_dev, void *stream) {
    if (ctx && !ctx->broken && n_inst == 0) return JACPCG_OK;   // an empty batch
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    jacpcg_plan *pl = nullptr;
    jacpcg_status st =
        make_plan(ctx, inst, n_inst, status_dev, iters_dev, resid_dev, beta_dev, 0, s, &pl);
    if (st != JACPCG_OK) return st;
    st = execute(pl, s);
    drop_plan(pl);
    return st;
}

jacpcg_status jacpcg_plan_bytes(const jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst,
                                size_t *bytes) {
    if (!bytes) return JACPCG_EINVAL;
    jacpcg_status st = validate(ctx, inst, n_inst);
    if (st != JACPCG_OK) return st;
    *bytes = align_up(make_layout(ctx->cfg, inst, n_inst, ctx->cfg.refine_sweeps > 0, ctx->pcg_shape_idx).total);
    return JACPCG_OK;
}

jacpcg_status jacpcg_arena_free_bytes(const jacpcg_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return JACPCG_EINVAL;
    size_t s = ctx->arena.free_bytes();
    for (auto &p : ctx->arena.pending) s += p.bytes;
    *bytes = s;
    return JACPCG_OK;
}

jacpcg_status jacpcg_profile_read(jacpcg_ctx *ctx, float ms[4], int *n_executes,
                                  int *launches_per_execute) {
    if (!ctx || !ms) return JACPCG_EINVAL;
    for (int i = 0; i < 4; ++i) ms[i] = 0.f;
    for (size_t k = 0; k < ctx->prof_used; ++k) {
        auto &ev = ctx->prof_pool[k];
        if (cudaEventSynchronize(ev[4]) != cudaSuccess) return cuda_fail(ctx);
        for (int i = 0; i < 4; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) != cudaSuccess) return cuda_fail(ctx);
            ms[i] += t;
        }
    }
    if (n_executes) *n_executes = (int)ctx->prof_used;
    if (launches_per_execute) *launches_per_execute = ctx->last_launches;
    ctx->prof_used = 0;
    return JACPCG_OK;
}

int64_t jacpcg_launch_count(const jacpcg_ctx *ctx) { return ctx ? ctx->launches : -1; }

const char *jacpcg_last_cuda_error(const jacpcg_ctx *ctx) {
    if (!ctx) return "no context";
    return ctx->broken ? cudaGetErrorString(ctx->last_error) : "no error";
}

jacpcg_status jacpcg_set_shape(jacpcg_ctx *ctx, int k_class_, int shape) {
    if (!ctx || k_class_ < 8 || k_class_ > 256 || (k_class_ & (k_class_ - 1))) return JACPCG_EINVAL;
    const int c = kc_index(k_class_);
    if (shape < -1 || shape >= PCG_NSHAPES[c]) return JACPCG_EINVAL;
    ctx->pcg_shape_idx[c] = shape;
    return JACPCG_OK;
}

jacpcg_status jacpcg_get_shape(const jacpcg_ctx *ctx, int k_class_, int *shape, int *n_shapes,
                               int *cols_per_warp, int *warps_per_cta) {
    if (!ctx || k_class_ < 8 || k_class_ > 256 || (k_class_ & (k_class_ - 1))) return JACPCG_EINVAL;
    const int c = kc_index(k_class_);
    const bool tensor = ctx->pcg_shape_idx[c] < 0 && tensor_iteration_allowed(ctx->cfg, k_class_);
    const PcgShape s = pcg_shape(k_class_, ctx->pcg_shape_idx[c]);
    if (shape) *shape = tensor ? -1 : (ctx->pcg_shape_idx[c] < 0 ? 0 : ctx->pcg_shape_idx[c]);
    if (n_shapes) *n_shapes = PCG_NSHAPES[c];
    if (cols_per_warp) *cols_per_warp = s.CW;
    if (warps_per_cta) *warps_per_cta = s.NW;
    return JACPCG_OK;
}

jacpcg_status jacpcg_autotune(jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst, void *stream,
                              char *table, size_t table_cap) {
    jacpcg_status st = validate(ctx, inst, n_inst);
    if (st != JACPCG_OK) return st;
    if (ctx->broken) return JACPCG_ECUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_fail(ctx);
    std::string js = "{";
    bool first = true;
    for (int KC : {8, 16, 32, 64, 128, 256}) {
        std::vector<jacpcg_instance> sub;
        for (int i = 0; i < n_inst; ++i)
            if (k_class(inst[i].K) == KC) sub.push_back(inst[i]);
        if (sub.empty()) continue;
        const int c = kc_index(KC);
        float best_ms = 1e30f;
        int best = 0;
        std::string times;
        const int first_sh = tensor_iteration_allowed(ctx->cfg, KC) ? -1 : 0;   // -1: tensor cores
        for (int sh = first_sh; sh < PCG_NSHAPES[c] && st == JACPCG_OK; ++sh) {
            ctx->pcg_shape_idx[c] = sh;
            jacpcg_plan *pl = nullptr;
            st = make_plan(ctx, sub.data(), (int)sub.size(), nullptr, nullptr, nullptr, nullptr, 0, nullptr, &pl);
            if (st != JACPCG_OK) break;
            float ms = 0.f;
            for (int r = 0; r < 2 && st == JACPCG_OK; ++r) st = execute(pl, s);
            if (st == JACPCG_OK && cudaEventRecord(e0, s) != cudaSuccess) st = cuda_fail(ctx);
            for (int r = 0; r < 5 && st == JACPCG_OK; ++r) st = execute(pl, s);
            if (st == JACPCG_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                st = cuda_fail(ctx);
            drop_plan(pl);
            ms /= 5.f;
            if (st == JACPCG_OK && ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
            times += (sh != first_sh ? ", " : "") + std::to_string(ms);
        }
        ctx->pcg_shape_idx[c] = best;
        const PcgShape b = pcg_shape(KC, best);
        js += (first ? "" : ", ") + std::string("\"") + std::to_string(KC) + "\": {\"shape\": " + std::to_string(best) +
              ", \"path\": \"" + (best < 0 ? "tensor" : "simt") + "\"" +
              ", \"cols_per_warp\": " + std::to_string(best < 0 ? 0 : b.CW) +
              ", \"warps_per_cta\": " + std::to_string(best < 0 ? 0 : b.NW) +
              ", \"instances\": " + std::to_string(sub.size()) +
              ", \"candidates\": [" + (first_sh < 0 ? "\"tensor\", " : "") + "\"simt shapes 0.." +
              std::to_string(PCG_NSHAPES[c] - 1) + "\"]" + ", \"ms_per_candidate\": [" + times + "]}";
        first = false;
        if (st != JACPCG_OK) break;
    }
    js += "}";
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (table && table_cap > 0) {
        const size_t n = js.size() < table_cap - 1 ? js.size() : table_cap - 1;
        std::memcpy(table, js.data(), n);
        table[n] = 0;
    }
    return st;
}

}  // extern "C"
