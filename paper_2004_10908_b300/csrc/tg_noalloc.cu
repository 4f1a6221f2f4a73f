// tg_noalloc.cu -- tg_run_noalloc: run one graph without allocating anything.
//
// Some callers cannot allocate device memory at all: code running inside
// another framework's memory pool that forbids cudaMalloc, plugins handed
// only pre-allocated buffers, or hosts that must not change the device's
// memory footprint after start-up.  For them this entry point keeps all of
// its scratch memory (packed task records, join words, ready queues,
// descriptors, counters) in ONE file-scope __device__ array of a fixed size.
// The array exists on every GPU that loads the library until the process
// exits.  The caller passes device pointers to its inputs and outputs.
//
// Limits: at most kNaMaxNodes tasks and kNaMaxEdges edges per call; the
// array holds kScratchBytes = 6,892,032 bytes (about 6.6 MiB).
// Every call shares the array: calls that overlap on the GPU (from several
// host threads or streams) race and corrupt each other.  The first call on
// a device looks up the array's device address (cudaGetSymbolAddress) and
// configures the kernel.  No call can be made while its stream is being
// captured into a CUDA graph: every call synchronises the stream and reads
// status words back to the host.
#include <cstring>
#include <mutex>

#include "../../include/tg.h"
#include "tg_internal.h"

namespace tg {
namespace {

constexpr u32 kNaMaxNodes = 1u << 16;
constexpr u32 kNaMaxEdges = 1u << 18;
constexpr u32 kNaMaxBlocks = 160;
constexpr u32 kNaWarps = 8;
constexpr u32 kNaDequeDepth = 1024;
constexpr u32 kNaRing = 1024;
constexpr u32 kNaThieves = 16;
constexpr u32 kNaInjCap = 1u << 17;   // power of two >= kNaMaxNodes + 4096
constexpr int kNaMaxDevices = 64;

// byte offsets inside the scratch array (each region 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffStats = al(kOffCtl + sizeof(LaunchCtl));
constexpr size_t kOffThief = al(kOffStats + (size_t)kNaMaxBlocks * ST_COUNT * 8);
constexpr size_t kOffDesc = al(kOffThief + (size_t)kNaThieves * 128);
constexpr size_t kOffWords = al(kOffDesc + sizeof(GDesc));   // status / counters
constexpr size_t kOffDqc = al(kOffWords + 256);
constexpr size_t kOffDq = al(kOffDqc + (size_t)kNaMaxBlocks * sizeof(QCtr));
constexpr size_t kOffInj = al(kOffDq + (size_t)kNaMaxBlocks * kNaDequeDepth * 8);
constexpr size_t kOffSlots = al(kOffInj + (size_t)kNaInjCap * 8);
constexpr size_t kOffOut = al(kOffSlots + (size_t)kNaMaxNodes * sizeof(NodeSlot));
constexpr size_t kOffGid = al(kOffOut + (size_t)kNaMaxNodes * 4);
constexpr size_t kOffEdges = al(kOffGid + (size_t)kNaMaxNodes * 4);
constexpr size_t kOffStrong = al(kOffEdges + ((size_t)kNaMaxEdges + kNaMaxNodes) * 4);
constexpr size_t kOffWeak = al(kOffStrong + (size_t)kNaMaxNodes * 4);
constexpr size_t kScratchBytes = al(kOffWeak + (size_t)kNaMaxNodes * 4);

// The scratch memory itself.
static_assert(kScratchBytes == 6892032, "the stated size of the scratch array must follow its layout");
static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

// words at kOffWords
enum { W_STATUS = 0, W_NSRC = 1, W_FINAL = 2 };

struct NaDevice {
    bool ready = false;
    unsigned char *base = nullptr;
    int blocks = 0;
};
NaDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mu;

__device__ __forceinline__ void na_fail(i32 *status, i32 code) { atomicCAS(status, 0, code); }

// Pass 1: validate tasks and edges; count strong and weak in-degrees.
__global__ void na_count_kernel(u32 n, u32 m, const u8 *kinds, const u32 *params, const u32 *succ_off,
                                const u32 *succ, unsigned char *base)
{
    i32 *words = (i32 *)(base + kOffWords);
    u32 *strong = (u32 *)(base + kOffStrong);
    u32 *weak = (u32 *)(base + kOffWeak);
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const u32 kind = kinds[v];
        const u32 a = succ_off[v], b = succ_off[v + 1];
        if (kind > TG_COND_CONST || b < a || b > m || b - a > 0xFFFFu ||
            (kind == TG_COND_LOOP && ((params[v] >> 16) & 0xFFu) == 0u) || (kind != TG_STATIC && a == b)) {
            na_fail(&words[W_STATUS], TG_ERR_INVALID);
            continue;
        }
        for (u32 e = a; e < b; ++e) {
            const u32 t = succ[e];
            if (t >= n) {
                na_fail(&words[W_STATUS], TG_ERR_INVALID);
                break;
            }
            atomicAdd(kind == TG_STATIC ? &strong[t] : &weak[t], 1u);
        }
    }
}

// Pass 2: pack the 32-byte task records, the successor lists and the sources.
__global__ void na_pack_kernel(u32 n, u32 m, const u8 *kinds, const u32 *params, const u32 *succ_off,
                               const u32 *succ, u32 seed, unsigned char *base)
{
    i32 *words = (i32 *)(base + kOffWords);
    const u32 *strong = (const u32 *)(base + kOffStrong);
    const u32 *weak = (const u32 *)(base + kOffWeak);
    NodeSlot *slots = (NodeSlot *)(base + kOffSlots);
    u32 *gidv = (u32 *)(base + kOffGid);
    u32 *edges = (u32 *)(base + kOffEdges);
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const u32 kind = kinds[v];
        const u32 a = succ_off[v], b = succ_off[v + 1];
        if (b < a || b > m)
            continue;   // reported by the counting pass
        if (strong[v] > 0xFFFFu)
            na_fail(&words[W_STATUS], TG_ERR_INVALID);
        u32 arg = 0;
        if (kind == TG_COND_LOOP)
            arg = (params[v] >> 16) & 0xFFu;
        else if (kind == TG_COND_CONST)
            arg = params[v] >> 24;
        NodeSlot s;
        s.succ_off = a;
        s.deg = (b - a) | (strong[v] << 16);
        s.prm = (params[v] & 0xFFFFu) | (kind << 16) | (arg << 24);
        s.lid = v;
        s.W = strong[v];
        s.cnt = 0;
        s.dig = 0;
        slots[v] = s;
        gidv[v >> kChunkShift] = 0;
        for (u32 e = a; e < b; ++e) {
            const u32 t = succ[e];
            edges[e] = t | ((kind == TG_STATIC && t < n && strong[t] == 1u) ? kSoleBit : 0u);
        }
        if (strong[v] == 0 && weak[v] == 0) {
            u32 k = atomicAdd((u32 *)&words[W_NSRC], 1u);
            edges[m + k] = v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        GDesc *d = (GDesc *)(base + kOffDesc);
        d->seed = seed;
        d->node_off = 0;
        d->n = n;
        d->src_off = m;
        d->exec_cap = 1u << 31;
    }
}

// After packing: the source count (every thread of pass 2 is done) and the
// offsets' end, which must equal the edge count.
__global__ void na_sources_kernel(u32 n, u32 m, const u32 *succ_off, unsigned char *base)
{
    i32 *words = (i32 *)(base + kOffWords);
    GDesc *d = (GDesc *)(base + kOffDesc);
    if (succ_off[n] != m)
        na_fail(&words[W_STATUS], TG_ERR_INVALID);
    d->n_src = (u32)words[W_NSRC];
    if (words[W_NSRC] == 0)
        na_fail(&words[W_STATUS], TG_ERR_NO_SOURCE);
}

// Copy the per-task results into the caller's output arrays.
__global__ void na_gather_kernel(u32 n, unsigned char *base, u32 *out, u32 *cnt, u32 *dig)
{
    const NodeSlot *slots = (const NodeSlot *)(base + kOffSlots);
    const u32 *outv = (const u32 *)(base + kOffOut);
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (out)
            out[v] = outv[v];
        if (cnt)
            cnt[v] = slots[v].cnt & ~(kInflight | kAwait);
        if (dig)
            dig[v] = slots[v].dig;
    }
}

// Once per device, with that device current: find the scratch array's device
// address and configure the scheduler for this launch shape.
int na_setup(int dev, NaDevice **out)
{
    std::lock_guard<std::mutex> lk(g_na_mu);
    NaDevice &d = g_na_dev[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess || !ptr)
            return TG_ERR_CUDA;
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return TG_ERR_CUDA;
        if (sched_occupancy((int)(kNaWarps * 32), sched_dyn_smem(kNaRing, kNaWarps), &per_sm) != cudaSuccess ||
            per_sm <= 0)
            return TG_ERR_CUDA;
        d.base = (unsigned char *)ptr;
        d.blocks = sms < (int)kNaMaxBlocks ? sms : (int)kNaMaxBlocks;
        d.ready = true;
    }
    *out = &d;
    return TG_OK;
}

}  // namespace
}  // namespace tg

using namespace tg;

extern "C" int tg_run_noalloc(uint32_t n_nodes, const uint8_t *kinds, const uint32_t *params,
                              const uint32_t *succ_off, const uint32_t *succ, uint32_t n_edges, uint32_t seed,
                              uint32_t *out, uint32_t *cnt, uint32_t *dig, void *cuda_stream)
{
    if (n_nodes == 0 || !kinds || !params || !succ_off || (n_edges && !succ))
        return TG_ERR_INVALID;
    if (n_nodes > kNaMaxNodes || n_edges > kNaMaxEdges)
        return TG_ERR_BUDGET;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
        return TG_ERR_CUDA;
    NaDevice *d = nullptr;
    int rc = na_setup(dev, &d);
    if (rc != TG_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char *base = d->base;

    // the last call's contents stay in the array: zero what must start at zero
    if (cudaMemsetAsync(base + kOffWords, 0, 256, st) != cudaSuccess ||
        cudaMemsetAsync(base + kOffStrong, 0, (size_t)n_nodes * 4, st) != cudaSuccess ||
        cudaMemsetAsync(base + kOffWeak, 0, (size_t)n_nodes * 4, st) != cudaSuccess ||
        cudaMemsetAsync(base + kOffDesc, 0, sizeof(GDesc), st) != cudaSuccess ||
        cudaMemsetAsync(base + kOffThief, 0, (size_t)kNaThieves * 128, st) != cudaSuccess)
        return TG_ERR_CUDA;
    if (launch_clear((u64 *)(base + kOffInj), kNaInjCap, st) != cudaSuccess ||
        launch_clear((u64 *)(base + kOffDq), (size_t)d->blocks * kNaDequeDepth, st) != cudaSuccess)
        return TG_ERR_CUDA;
    const u32 grid = (n_nodes + 255u) / 256u;
    na_count_kernel<<<grid, 256, 0, st>>>(n_nodes, n_edges, kinds, params, succ_off, succ, base);
    na_pack_kernel<<<grid, 256, 0, st>>>(n_nodes, n_edges, kinds, params, succ_off, succ, seed, base);
    na_sources_kernel<<<1, 1, 0, st>>>(n_nodes, n_edges, succ_off, base);
    if (cudaGetLastError() != cudaSuccess)
        return TG_ERR_CUDA;
    i32 words[2] = {0, 0};
    if (cudaMemcpyAsync(words, base + kOffWords, sizeof(words), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TG_ERR_CUDA;
    if (words[W_STATUS] != 0)
        return words[W_STATUS];

    KParams p{};
    p.slots = (NodeSlot *)(base + kOffSlots);
    p.outv = (u32 *)(base + kOffOut);
    p.chunk_gid = (const u32 *)(base + kOffGid);
    p.edges = (const u32 *)(base + kOffEdges);
    p.descs = (GDesc *)(base + kOffDesc);
    p.lt = nullptr;
    p.n_graphs = 1;
    p.single_gid = 0;
    p.max_n = n_nodes;
    p.total_sources = (u32)words[W_NSRC];
    p.ctl = (LaunchCtl *)(base + kOffCtl);
    p.stats = (u64 *)(base + kOffStats);
    p.inj = (u64 *)(base + kOffInj);
    p.inj_mask = kNaInjCap - 1u;
    p.nblocks = (u32)d->blocks;
    p.dq = (u64 *)(base + kOffDq);
    p.dqc = (QCtr *)(base + kOffDqc);
    p.dq_mask = kNaDequeDepth - 1u;
    p.dq_stride = kNaDequeDepth;
    p.batch_max = 32;
    p.smem_mask = kNaRing - 1u;
    p.flags = 0;
    p.max_steal = 8;
    p.steal_policy = 0;
    p.node_cap = kNaMaxNodes;
    p.idle_sleep_ns = 256;
    p.steal_backoff_ns = 512;
    p.keep_idle = 0;
    p.hand_batch = 0;
    p.max_thieves = kNaThieves;
    p.thief_slots = (u32 *)(base + kOffThief);
    p.time_limit_ns = 10ull * 1000 * 1000 * 1000;
    p.cancel = nullptr;
    p.status_out = (i32 *)(base + kOffWords) + W_FINAL;
    if (launch_rearm(p, st) != cudaSuccess || launch_sched(p, d->blocks, (int)(kNaWarps * 32), st) != cudaSuccess ||
        launch_finalize(p, st) != cudaSuccess)
        return TG_ERR_CUDA;
    na_gather_kernel<<<grid, 256, 0, st>>>(n_nodes, base, out, cnt, dig);
    if (cudaGetLastError() != cudaSuccess)
        return TG_ERR_CUDA;
    i32 final_status = 0;
    if (cudaMemcpyAsync(&final_status, base + kOffWords + W_FINAL * sizeof(i32), sizeof(i32),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TG_ERR_CUDA;
    return final_status;
}
