// noalloc.cu -- jacpcg_precode_noalloc: the batched precoder for callers
// that cannot allocate memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: real-time
// slot loops that forbid allocator latency and fragmentation, and embedded
// integrations whose memory was fixed at start-up.  This entry point
// allocates nothing, on the device or on the host: the instance table, tile
// lists, per-instance accumulators and the Gram / iterate workspace all live
// in one file-scope __device__ array of JACPCG_NOALLOC_SCRATCH_BYTES (every
// GPU that loads the library holds it until the process exits).  The tables
// are built in a file-scope static host array and reach the device as the
// by-value parameters of small upload kernels (no host-to-device copy, so
// the host never waits on the stream).  It runs the same kernels as
// jacpcg_precode, with each K class's default launch shape.
//
// The array's name in host code is a host-side stand-in, not a device
// address, so its device address is looked up with cudaGetSymbolAddress
// once per device, with that device current (the first call on a device
// does this set-up; make that first call before any stream capture), and
// passed to the kernels.  The lookup is repeated when the device's context
// is replaced (cudaDeviceReset reloads the module at a new address).
// Every call shares the array and the array keeps the last call's contents;
// the per-instance accumulators are reset by the first kernel of each call.
// Calls whose GPU work overlaps (two streams, or two threads) race on the
// array: serialise them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/jacpcg.h"
#include "common.cuh"
#include "kernels.h"

using namespace jacpcg;

namespace {

constexpr size_t kScratchBytes = JACPCG_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTableBytes = 256 * 1024;   // host image of the tables
constexpr int kMaxDevices = 64;
constexpr size_t kAlign = 256;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

alignas(256) unsigned char g_host_tables[kTableBytes];
void *g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];   // id of the context the address belongs to
std::mutex g_mutex;

// Tables travel as kernel parameters: each launch carries kChunk bytes by
// value and copies them into the scratch array.
constexpr int kChunk = 16 * 1024;
struct TableChunk {
    alignas(16) unsigned char bytes[kChunk];
};
static_assert(sizeof(TableChunk) + 32 <= 32764, "kernel parameter limit");
__global__ void __launch_bounds__(256) upload_tables(const __grid_constant__ TableChunk c, char *dst, int n) {
    const int4 *src = reinterpret_cast<const int4 *>(c.bytes);
    int4 *out = reinterpret_cast<int4 *>(dst);
    for (int i = threadIdx.x; i < n / 16; i += blockDim.x) out[i] = src[i];
}

// The unique id of the current context (cuCtxGetCurrent + cuCtxGetId through
// the runtime's driver entry points; no link against the driver library).
bool current_context_id(unsigned long long &id) {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1{}, q2{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return false;
        get_current = reinterpret_cast<GetCurrent>(f1);
        get_id = reinterpret_cast<GetId>(f2);
    }
    CUcontext ctx = nullptr;
    return get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS;
}

size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int kclass(int K) {
    int c = 8;
    while (c < K) c <<= 1;
    return c;
}
bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int gram_tiles(int KC) {
    const int nb = std::max(1, KC / gram_tb(KC));
    return nb * (nb + 1) / 2;
}
int pcg_blocks(int K) {
    const PcgShape s = pcg_shape(kclass(K));
    return (K + s.CW * s.NW - 1) / (s.CW * s.NW);
}
int w_tiles(int M, int K) {
    const int TN = hx_tn(kclass(K));
    return ((M + HX_TM - 1) / HX_TM) * ((K + TN - 1) / TN);
}
size_t ws_bytes(int M, int K) {
    const size_t KC = kclass(K);
    return 2 * up(KC * KC * sizeof(float2)) + up(KC * sizeof(float)) + up(w_tiles(M, K) * sizeof(float));
}

}  // namespace

extern "C" jacpcg_status jacpcg_precode_noalloc(const jacpcg_instance *inst, int n_inst,
                                                int variant, int32_t *status_dev,
                                                int32_t *iters_dev, float *resid_dev,
                                                float *beta_dev, void *stream) {
    if (!inst || n_inst < 1 || variant < JACPCG_STANDARD || variant > JACPCG_CG)
        return JACPCG_EINVAL;
    for (int i = 0; i < n_inst; ++i) {
        const jacpcg_instance &q = inst[i];
        if (q.K < 1 || q.K > 256 || q.M < 1) return JACPCG_EINVAL;
        if (q.ldh < q.M || q.ldw < q.M || (q.ldh & 1) || (q.ldw & 1)) return JACPCG_EINVAL;
        if (!q.H || !q.W || !al16(q.H) || !al16(q.W)) return JACPCG_EINVAL;
        if ((q.X && !al16(q.X)) || (q.A && !al16(q.A))) return JACPCG_EINVAL;
        if (!std::isfinite(q.xi) || q.xi < 0.0 || (q.K > q.M && !(q.xi > 0.0))) return JACPCG_EINVAL;
        if (!std::isfinite(q.power) || !std::isfinite(q.tol)) return JACPCG_EINVAL;
        if (q.max_iter < 0 || q.max_iter > 4096) return JACPCG_EINVAL;
        if (q.h_dtype != JACPCG_H_C64) return JACPCG_EINVAL;   // complex64 H only
        if (q.B || q.X0) return JACPCG_EINVAL;                // B = I, zero start only
        if (q.sinr) return JACPCG_EINVAL;                     // no SINR output here
    }
    // sizes: tables, accumulators, workspace -- all must fit the static arrays
    size_t ng = 0, np = 0, nh = 0, ws = 0;
    for (int i = 0; i < n_inst; ++i) {
        ng += gram_tiles(kclass(inst[i].K));
        np += pcg_blocks(inst[i].K);
        nh += w_tiles(inst[i].M, inst[i].K);
        ws += ws_bytes(inst[i].M, inst[i].K);
    }
    const size_t o_insts = 0;
    const size_t o_gram = o_insts + up(sizeof(DevInst) * n_inst);
    const size_t o_pcg = o_gram + up(sizeof(int4) * ng);
    const size_t o_hx = o_pcg + up(sizeof(int2) * np);
    const size_t o_acc = o_hx + up(sizeof(int4) * nh);
    const size_t o_ws = o_acc + 3 * up(sizeof(int32_t) * n_inst);
    if (o_acc > kTableBytes || o_ws + ws > kScratchBytes) return JACPCG_ENOMEM;

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return JACPCG_ECUDA;
    }
    // once per device (and again if its context was replaced), with that
    // device current; the runtime call itself makes the primary context current
    unsigned long long ctx_id = 0;
    const bool have_ctx = current_context_id(ctx_id);
    if (!g_scratch_addr[dev] || !have_ctx || g_scratch_ctx[dev] != ctx_id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return JACPCG_ECUDA;
        }
        if (!current_context_id(ctx_id)) return JACPCG_ECUDA;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx_id;
    }
    char *base = static_cast<char *>(g_scratch_addr[dev]);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);

    // host image of the tables, pointing into the device scratch
    DevInst *hi = reinterpret_cast<DevInst *>(g_host_tables + o_insts);
    size_t w = o_ws;
    for (int i = 0; i < n_inst; ++i) {
        const jacpcg_instance &q = inst[i];
        const int KC = kclass(q.K);
        char *b = base + w;
        DevInst d{};
        d.H = static_cast<const float2 *>(q.H);
        d.W = static_cast<float2 *>(q.W);
        d.Xout = static_cast<float2 *>(q.X);
        d.Aout = static_cast<float2 *>(q.A);
        d.A = reinterpret_cast<float2 *>(b);
        d.X = reinterpret_cast<float2 *>(b + up((size_t)KC * KC * sizeof(float2)));
        d.dinv = reinterpret_cast<float *>(b + 2 * up((size_t)KC * KC * sizeof(float2)));
        d.wpart = reinterpret_cast<float *>(b + 2 * up((size_t)KC * KC * sizeof(float2)) +
                                            up(KC * sizeof(float)));
        d.M = q.M; d.K = q.K; d.ldh = q.ldh; d.ldw = q.ldw; d.KC = KC;
        d.ncols = q.K;   // B = I
        d.max_iter = q.max_iter;
        d.n_wpart = w_tiles(q.M, q.K);
        d.variant = variant;
        d.xi = (float)q.xi;
        d.power = q.power > 0.0 ? (float)q.power : 1.0f;
        d.tol = q.tol;
        hi[i] = d;
        w += ws_bytes(q.M, q.K);
    }
    struct Group {
        int kind, param, first, count;
    } groups[12];
    int ngroups = 0;
    int4 *gt = reinterpret_cast<int4 *>(g_host_tables + o_gram);
    int g = 0;
    for (int TB : {16, 32, 64}) {
        const int start = g;
        for (int i = 0; i < n_inst; ++i) {
            const int KC = kclass(inst[i].K);
            if (gram_tb(KC) != TB) continue;
            const int nb = std::max(1, KC / TB);
            for (int bi = 0; bi < nb; ++bi)
                for (int bj = 0; bj <= bi; ++bj) gt[g++] = make_int4(i, bi, bj, 0);
        }
        if (g > start) groups[ngroups++] = {0, TB, start, g - start};
    }
    int2 *pb = reinterpret_cast<int2 *>(g_host_tables + o_pcg);
    int p = 0;
    for (int KC : {8, 16, 32, 64, 128, 256}) {
        const int start = p;
        const PcgShape sh = pcg_shape(KC);
        for (int i = 0; i < n_inst; ++i) {
            if (kclass(inst[i].K) != KC) continue;
            for (int c0 = 0; c0 < inst[i].K; c0 += sh.CW * sh.NW) pb[p++] = make_int2(i, c0);
        }
        if (p > start) groups[ngroups++] = {1, KC, start, p - start};
    }
    int4 *ht = reinterpret_cast<int4 *>(g_host_tables + o_hx);
    int h = 0;
    for (int TN : {16, 32, 64}) {
        const int start = h;
        for (int i = 0; i < n_inst; ++i) {
            if (hx_tn(kclass(inst[i].K)) != TN) continue;
            const int nm = (inst[i].M + HX_TM - 1) / HX_TM, nn = (inst[i].K + TN - 1) / TN;
            int slot = 0;
            for (int nt = 0; nt < nn; ++nt)
                for (int mt = 0; mt < nm; ++mt) ht[h++] = make_int4(i, mt, nt, slot++);
        }
        if (h > start) groups[ngroups++] = {2, TN, start, h - start};
    }
    // the tables as kernel parameters, kChunk bytes per launch (o_acc is a
    // multiple of 256, so every chunk is a whole number of 16-byte words)
    for (size_t off = 0; off < o_acc; off += kChunk) {
        const int n = (int)std::min<size_t>(kChunk, o_acc - off);
        TableChunk c;
        std::memcpy(c.bytes, g_host_tables + off, n);
        upload_tables<<<1, 256, 0, s>>>(c, base + off, n);
    }
    if (cudaGetLastError() != cudaSuccess) return JACPCG_ECUDA;
    const DevInst *d_insts = reinterpret_cast<const DevInst *>(base + o_insts);
    DevAccum acc;
    acc.flags = reinterpret_cast<int32_t *>(base + o_acc);
    acc.iters = reinterpret_cast<int32_t *>(base + o_acc + up(sizeof(int32_t) * n_inst));
    acc.resid_bits = reinterpret_cast<uint32_t *>(base + o_acc + 2 * up(sizeof(int32_t) * n_inst));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < ngroups && e == cudaSuccess; ++k) {
        const Group &G = groups[k];
        if (G.kind == 0)
            e = launch_gram_simt(G.param, d_insts,
                                 reinterpret_cast<const int4 *>(base + o_gram) + G.first, G.count, acc, s);
        else if (G.kind == 1)
            e = launch_pcg(G.param, variant, d_insts,
                           reinterpret_cast<const int2 *>(base + o_pcg) + G.first, G.count, acc, s);
        else
            e = launch_hx_simt(G.param, d_insts, reinterpret_cast<const int4 *>(base + o_hx) + G.first,
                               G.count, s);
    }
    if (e == cudaSuccess)
        e = launch_finalize(d_insts, n_inst, acc, DevOut{status_dev, iters_dev, resid_dev, beta_dev}, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return JACPCG_ECUDA;
    }
    return JACPCG_OK;
}
