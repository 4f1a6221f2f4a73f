// tg_host.cpp -- host side of libtg: context and arena pools, graph ingest /
// validation / CSR packing (strong/weak rule of "Scheduling Condition Tasks",
// source set of Algorithm 8), launches, batches and tickets.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <functional>
#include <map>
#include <set>
#include <new>
#include <vector>

#include "../../include/tg.h"
#include "tg_internal.h"

#if defined(__x86_64__)
#include <emmintrin.h>
#endif

using namespace tg;

namespace {

constexpr u32 kMaxGraphs = 1u << 16;
constexpr u32 kMaxDegree = 0xFFFFu;
constexpr int kMaxBlocks = 1024;   // per-block structures are allocated for this many blocks
constexpr u32 kSubRing = 1u << 16;  // server-mode submission / completion ring entries

// Launch geometry of the persistent scheduler: chosen per launch (a batch
// keeps the one it was captured with), within what the context allocated.
struct Geometry {
    int blocks = 0, threads = 0;
    u32 ring = 0, depth = 0, policy = 0, max_steal = 0, thieves = 0, idle_ns = 0, batch = 32, keep = 0, tmode = 0,
        backoff = 512, keep_idle = 0, hand_batch = 0;
};

u64 now_ns()
{
    return (u64)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

u64 next_pow2(u64 x)
{
    u64 p = 1;
    while (p < x)
        p <<= 1;
    return p;
}

bool is_pow2(u64 x) { return x && !(x & (x - 1)); }

// First-fit range allocator over [0, cap).
struct RangeAlloc {
    std::map<u64, u64> free_;   // start -> length
    u64 cap = 0;

    void init(u64 c)
    {
        cap = c;
        free_.clear();
        if (c)
            free_[0] = c;
    }
    bool alloc(u64 n, u64 &off)
    {
        if (n == 0) {
            off = 0;
            return true;
        }
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                u64 rest = it->second - n;
                free_.erase(it);
                if (rest)
                    free_[off + n] = rest;
                return true;
            }
        }
        return false;
    }
    void release(u64 off, u64 n)
    {
        if (n == 0)
            return;
        auto it = free_.emplace(off, n).first;
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
};

}  // namespace

// A graph owns its packed form in the edge pool -- successor lists (graph-
// local ids) and the source list -- and an execution instance: a chunk-
// aligned range of the node pool (task records + join/execution state +
// outputs) and a descriptor slot (gid).  An instance made by
// tg_instance_create shares its template's packed form and owns only an
// execution range and a gid; its records are re-armed from the immutable
// half of the template's own records.
struct tg_graph {
    tg_ctx *ctx = nullptr;
    tg_graph *tmpl = nullptr;     // the graph whose packed form this instance uses
    int n_inst = 0;               // live instances made from this graph
    u32 gid = 0;
    u32 n = 0, m = 0, n_src = 0, n_cond = 0;
    u64 node_off = 0, chunk_off = 0, n_chunks = 0;
    u64 edge_off = 0, edge_len = 0;
    u32 seed = 0;
    u64 pack_ns = 0, upload_ns = 0, bytes = 0;
    cudaEvent_t busy = nullptr;   // event of the launch it is in (null: idle)
    cudaEvent_t ready = nullptr;  // instance set-up copies (null: nothing to wait for)
    u64 serve_ticket = 0;         // server mode: ticket of the submission in flight
    bool setup_pending = false;   // an instance whose descriptor / chunk table are not written yet
    cudaGraphExec_t cap_exec = nullptr;   // capturer baseline (Algorithm 1), built for cap_streams
    u32 cap_streams = 0;
    std::vector<tg_graph *> mods;         // graphs its module tasks compose (distinct)
    std::vector<tg_graph *> sub_insts;    // one copy of its template per subflow task
    Geometry geo;                         // launch geometry chosen for it (tg_graph_autotune)
    bool has_geo = false;
    u32 n_mod = 0;                        // module and subflow tasks
    int n_refs = 0;                       // graphs whose module tasks compose this one
    int n_batches = 0;                    // live batches holding it
};

struct tg_batch {
    tg_ctx *ctx = nullptr;
    std::vector<tg_graph *> gs;
    std::vector<tg_graph *> comp;   // graphs its members' module and subflow tasks reach
    bool has_mod = false;
    bool counted = false;           // its members count it (tg_graph::n_batches)
    bool acyclic = false;           // no member has condition, module or subflow tasks
    u64 lt_off = 0, lt_len = 0;
    u32 max_n = 0, total_src = 0;
    Geometry geo;
    KParams kp{};
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool launched = false;
};

struct Submission {
    tg_graph *g = nullptr;
    cudaEvent_t ev = nullptr;
    int status = TG_PENDING;
};

struct tg_ctx {
    int device = 0, sm_count = 0;
    std::string dev_name;               // the device's name (keys of the tuning cache)
    std::set<tg_graph *> live_graphs;   // freed with the context if the caller did not
    std::set<tg_batch *> live_batches;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    tg_ctx_opts opts{};
    char *arena = nullptr;
    size_t arena_bytes = 0;

    LaunchCtl *ctl = nullptr;
    u64 *stats = nullptr;
    GDesc *descs = nullptr;
    QCtr *dqc = nullptr;
    u64 *dq = nullptr;
    u64 *inj = nullptr;
    u32 *scratch = nullptr;
    u32 *thief_slots = nullptr;
    NodeSlot *slots = nullptr;
    u32 *outv = nullptr;
    u32 *chunk_gid = nullptr;
    u32 *edges = nullptr;
    u64 *trace = nullptr;          // per-task trace records (3 words per task)
    cudaStream_t side = nullptr;   // instance set-up and server submissions
    SubEntry *sub = nullptr;       // device submission ring
    SubEntry *h_sub = nullptr;     // pinned staging of submission entries
    u64 *h_comp = nullptr, *d_comp = nullptr;   // host-mapped completion ring
    u32 *h_stop = nullptr, *d_stop = nullptr;   // host-mapped stop flag
    u64 sub_seq = 0, comp_read = 0;
    tg_graph **by_gid = nullptr;   // serving: graph in flight per gid
    std::map<u64, int> serve_done; // serving: finished tickets -> status
    std::vector<u64> newly_done;   // serving: tickets finished by the last drain
    Geometry serve_geo;

    u64 node_cap = 0, edge_cap = 0, inj_cap = 0;
    RangeAlloc nodes, edge_pool;
    std::vector<u32> free_gids;
    u64 budget = 0, used = 0;

    Geometry geo;        // geometry of single-graph launches
    u32 dq_cap = 0;      // entries allocated per block deque
    Geometry last_geo;   // geometry of the last scheduler launch (statistics)

    u32 *h_cancel = nullptr, *d_cancel = nullptr;
    i32 *h_status = nullptr, *d_status = nullptr;
    char *h_stage = nullptr;
    size_t stage_bytes = 0;

    bool dirty = true;   // queue slots may hold stale entries: clear before the next launch
    bool serving = false; // a resident scheduler runs on the context stream
    u64 next_ticket = 1;
    std::map<u64, Submission> subs;
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
    bool timed = false;
    // tg_graph_create_dev: device scratch (grown on demand), the validation
    // words' pinned copy, events around the input copies and the pack
    char *pk_scratch = nullptr;
    size_t pk_bytes = 0;
    u32 *h_pkflags = nullptr;
    cudaEvent_t pk_ev[3] = {nullptr, nullptr, nullptr};
    // tg_result_copy: the packed counts and digests (grown on demand)
    u64 *d_rb = nullptr;
    size_t rb_bytes = 0;
};

namespace {

#define TG_CUDA(call)                       \
    do {                                    \
        cudaError_t e_ = (call);            \
        if (e_ != cudaSuccess)              \
            return TG_ERR_CUDA;             \
    } while (0)

KParams base_params(tg_ctx *c, const Geometry &g)
{
    KParams p{};
    p.slots = c->slots;
    p.outv = c->outv;
    p.chunk_gid = c->chunk_gid;
    p.edges = c->edges;
    p.descs = c->descs;
    p.ctl = c->ctl;
    p.stats = c->stats;
    p.inj = c->inj;
    p.inj_mask = (u32)(c->inj_cap - 1);
    p.nblocks = (u32)g.blocks;
    p.dq = c->dq;
    p.dqc = c->dqc;
    p.dq_mask = g.depth - 1u;
    p.dq_stride = c->dq_cap;
    p.smem_mask = g.ring - 1u;
    p.flags = c->opts.flags & ~kFlagAcyclic;
    p.max_steal = g.max_steal;
    p.steal_policy = g.policy;
    p.node_cap = (u32)c->node_cap;
    p.idle_sleep_ns = g.idle_ns;
    p.max_thieves = g.thieves;
    p.batch_max = g.batch;
    p.local_keep = g.keep;
    p.thief_mode = g.tmode;
    p.steal_backoff_ns = g.backoff;
    p.keep_idle = g.keep_idle;
    p.hand_batch = g.hand_batch;
    p.thief_slots = c->thief_slots;
    p.time_limit_ns = c->opts.time_limit_ns;
    p.cancel = c->d_cancel;
    p.status_out = c->d_status;
    p.trace = c->trace;
    p.sub = c->sub;
    p.sub_mask = kSubRing - 1u;
    p.comp_mask = kSubRing - 1u;
    p.comp = c->d_comp;
    return p;
}

int ensure_stage(tg_ctx *c, size_t bytes)
{
    if (c->stage_bytes >= bytes)
        return TG_OK;
    if (c->h_stage) {
        cudaStreamSynchronize(c->stream);   // read-backs
        cudaStreamSynchronize(c->side);     // graph uploads
        cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->stage_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 22);
    if (cudaHostAlloc((void **)&c->h_stage, want, cudaHostAllocDefault) != cudaSuccess)
        return TG_ERR_CUDA;
    c->stage_bytes = want;
    return TG_OK;
}

// A graph is busy while the event of its last launch has not completed.
bool graph_busy(tg_graph *g)
{
    if (!g->busy)
        return false;
    if (cudaEventQuery(g->busy) == cudaErrorNotReady)
        return true;
    g->busy = nullptr;
    return false;
}

void note_status(tg_ctx *c, int st)
{
    if (st == TG_ERR_TIMEOUT || st == TG_ERR_CANCELLED || st == TG_ERR_INTERNAL)
        c->dirty = true;
}

int clear_if_dirty(tg_ctx *c)
{
    if (!c->dirty)
        return TG_OK;
    TG_CUDA(launch_clear(c->inj, c->inj_cap, c->stream));
    TG_CUDA(launch_clear(c->dq, (size_t)kMaxBlocks * c->dq_cap, c->stream));
    c->dirty = false;
    return TG_OK;
}

// Validate the launch fields of `o` (0 = default) and size the grid from the
// occupancy of the scheduler kernel at that block shape.
int resolve_geometry(const tg_ctx *c, const tg_ctx_opts &o, Geometry &g)
{
    const int warps = o.warps_per_block > 0 ? o.warps_per_block : 16;
    const u32 ring = o.smem_ring > 0 ? (u32)o.smem_ring : 1024u;
    const u32 depth = o.deque_depth > 0 ? (u32)o.deque_depth : c->dq_cap;
    if (warps > 32 || !is_pow2(ring) || ring < 64 || ring > 8192 || !is_pow2(depth) || depth < 64 ||
        depth > c->dq_cap || o.steal_policy < 0 || o.steal_policy > 1 || o.max_thieves > 1024 ||
        o.max_steal < 0 || o.worker_blocks < 0 || o.batch_max < 0 || o.batch_max > 32 || o.local_keep < 0 ||
        (u32)o.local_keep > ring || o.thief_mode < 0 || o.thief_mode > 1 || o.steal_backoff_ns > 1000000u ||
        o.keep_idle < 0 || o.keep_idle > 1 || o.hand_batch < 0 || o.hand_batch > 1)
        return TG_ERR_INVALID;
    int per_sm = 0;
    if (sched_occupancy(warps * 32, sched_dyn_smem(ring, (u32)warps), &per_sm) != cudaSuccess || per_sm <= 0)
        return TG_ERR_INVALID;   // this block shape cannot be resident
    const int max_blocks = std::min(per_sm * c->sm_count, kMaxBlocks);
    g.blocks = o.worker_blocks > 0 ? std::min(o.worker_blocks, max_blocks) : max_blocks;
    g.threads = warps * 32;
    g.ring = ring;
    g.depth = depth;
    g.policy = (u32)o.steal_policy;
    g.max_steal = o.max_steal > 0 ? (u32)o.max_steal : 8u;
    g.thieves = o.max_thieves > 0 ? (u32)o.max_thieves : 16u;
    g.idle_ns = o.idle_sleep_ns > 0 ? o.idle_sleep_ns : 256u;
    g.batch = o.batch_max > 0 ? (u32)o.batch_max : 32u;
    // a short shared-memory backlog: ready work beyond it goes to the block's
    // public deque where idle warps of other blocks can take it
    g.keep = std::min<u32>(o.local_keep > 0 ? (u32)o.local_keep : 32u, ring);
    g.tmode = (u32)o.thief_mode;
    g.backoff = o.steal_backoff_ns > 0 ? o.steal_backoff_ns : 512u;
    g.keep_idle = (u32)o.keep_idle;
    g.hand_batch = (u32)o.hand_batch;
    return TG_OK;
}

void geometry_to_opts(const Geometry &g, tg_ctx_opts &o)
{
    o.worker_blocks = g.blocks;
    o.warps_per_block = g.threads / 32;
    o.deque_depth = (int32_t)g.depth;
    o.steal_policy = (int32_t)g.policy;
    o.max_steal = (int32_t)g.max_steal;
    o.smem_ring = (int32_t)g.ring;
    o.max_thieves = (int32_t)g.thieves;
    o.idle_sleep_ns = g.idle_ns;
    o.batch_max = (int32_t)g.batch;
    o.local_keep = (int32_t)g.keep;
    o.thief_mode = (int32_t)g.tmode;
    o.steal_backoff_ns = g.backoff;
    o.keep_idle = (int32_t)g.keep_idle;
    o.hand_batch = (int32_t)g.hand_batch;
}

}  // namespace

extern "C" {

const char *tg_strerror(int s)
{
    switch (s) {
    case TG_OK: return "ok";
    case TG_PENDING: return "pending";
    case TG_ERR_INVALID: return "invalid argument or graph";
    case TG_ERR_NO_SOURCE: return "no task with zero strong and zero weak in-edges";
    case TG_ERR_EDGE_KIND: return "explicit edge kind disagrees with the source task's kind";
    case TG_ERR_BUDGET: return "graph does not fit the memory budget";
    case TG_ERR_RACE: return "task race: activation of a task already queued or running";
    case TG_ERR_EXEC_LIMIT: return "execution cap exceeded";
    case TG_ERR_TIMEOUT: return "device time limit expired";
    case TG_ERR_CANCELLED: return "cancelled";
    case TG_ERR_CUDA: return "CUDA runtime error";
    case TG_ERR_INTERNAL: return "scheduler internal error (bounded wait gave up)";
    case TG_ERR_BUSY: return "graph already in flight";
    default: return "unknown status";
    }
}

int tg_ctx_create(void *dev_arena, size_t arena_bytes, void *cuda_stream, const tg_ctx_opts *opts,
                  tg_ctx **out)
{
    if (!out || !dev_arena || ((uintptr_t)dev_arena & 255u) != 0)
        return TG_ERR_INVALID;
    *out = nullptr;
    tg_ctx *c = new (std::nothrow) tg_ctx();
    if (!c)
        return TG_ERR_INVALID;
    if (opts)
        c->opts = *opts;
    tg_ctx_opts &o = c->opts;
    if (o.deque_depth <= 0)
        o.deque_depth = 4096;
    if (!is_pow2((u64)o.deque_depth) || o.deque_depth < 64 || o.deque_depth > (1 << 20)) {
        delete c;
        return TG_ERR_INVALID;
    }
    if (o.time_limit_ns == 0)
        o.time_limit_ns = 10ull * 1000 * 1000 * 1000;
    if (o.exec_cap == 0 || o.exec_cap > (1ull << 31))
        o.exec_cap = 1ull << 31;

    c->stream = (cudaStream_t)cuda_stream;
    c->arena = (char *)dev_arena;
    c->arena_bytes = arena_bytes;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
        delete c;
        return TG_ERR_CUDA;
    }
    c->dev_name = prop.name;
    c->dq_cap = (u32)o.deque_depth;
    int rg = resolve_geometry(c, o, c->geo);
    if (rg != TG_OK) {
        delete c;
        return rg;
    }
    geometry_to_opts(c->geo, o);

    // ---- carve the arena
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        off = (off + 255) & ~(size_t)255;
        char *p = c->arena + off;
        off += bytes;
        return p;
    };
    c->ctl = (LaunchCtl *)take(sizeof(LaunchCtl));
    c->stats = (u64 *)take((size_t)kMaxBlocks * ST_COUNT * sizeof(u64));
    c->scratch = (u32 *)take(4096);
    c->thief_slots = (u32 *)take((size_t)1024 * 128);
    c->sub = (SubEntry *)take((size_t)kSubRing * sizeof(SubEntry));
    c->descs = (GDesc *)take((size_t)kMaxGraphs * sizeof(GDesc));
    c->dqc = (QCtr *)take((size_t)kMaxBlocks * sizeof(QCtr));
    c->dq = (u64 *)take((size_t)kMaxBlocks * c->dq_cap * sizeof(u64));
    off = (off + 255) & ~(size_t)255;
    if (off >= arena_bytes) {
        delete c;
        return TG_ERR_INVALID;
    }
    size_t rest = arena_bytes - off - 4096;
    const bool traced = (o.flags & (TG_OPT_TRACE | TG_OPT_TRACE_TASKS)) != 0u;
    u64 ncap = o.max_nodes, ecap = o.max_edges;
    ncap &= ~(u64)(kChunk - 1);
    if (ncap == 0) {
        // per task: 36 B execution range + 8 B of injection queue; the edge
        // pool (successor lists and sources) takes the rest
        ncap = (rest / (traced ? 152 : 128)) & ~(u64)255;
        if (ncap > kMaxNodeIndex)
            ncap = kMaxNodeIndex & ~(u64)255;
    }
    if (ncap == 0 || ncap > kMaxNodeIndex) {
        delete c;
        return TG_ERR_INVALID;
    }
    u64 icap = next_pow2(ncap + 4096);
    size_t fixed = (size_t)ncap * (sizeof(NodeSlot) + 8 + (traced ? 24 : 0)) + (size_t)icap * 8 + 4096;
    if (fixed >= rest) {
        delete c;
        return TG_ERR_INVALID;
    }
    if (ecap == 0)
        ecap = std::min<u64>((rest - fixed) / 4, 0xFFFFFFF0ull);
    if ((size_t)ecap * 4 + fixed > rest || ecap == 0) {
        delete c;
        return TG_ERR_INVALID;
    }
    c->inj = (u64 *)take((size_t)icap * 8);
    if (traced)
        c->trace = (u64 *)take((size_t)ncap * 24);
    c->slots = (NodeSlot *)take((size_t)ncap * sizeof(NodeSlot));
    c->outv = (u32 *)take((size_t)ncap * 4);
    c->chunk_gid = (u32 *)take((size_t)(ncap >> kChunkShift) * 4 + 256);
    c->edges = (u32 *)take((size_t)ecap * 4);
    if (off > arena_bytes) {
        delete c;
        return TG_ERR_INVALID;
    }
    c->node_cap = ncap;
    c->edge_cap = ecap;
    c->inj_cap = icap;
    c->nodes.init(ncap >> kChunkShift);   // allocated in 256-task chunks
    c->edge_pool.init(ecap);
    c->budget = o.mem_budget_bytes ? o.mem_budget_bytes : (u64)ncap * 36 + (u64)ecap * 4;
    c->free_gids.reserve(kMaxGraphs);
    for (u32 g = kMaxGraphs; g-- > 0;)
        c->free_gids.push_back(g);

    if (cudaHostAlloc((void **)&c->h_cancel, 64, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->d_cancel, c->h_cancel, 0) != cudaSuccess ||
        cudaHostAlloc((void **)&c->h_status, kMaxGraphs * sizeof(i32), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->d_status, c->h_status, 0) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc((void **)&c->h_sub, (size_t)kSubRing * sizeof(SubEntry), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&c->h_comp, (size_t)kSubRing * 8, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->d_comp, c->h_comp, 0) != cudaSuccess ||
        cudaHostAlloc((void **)&c->h_stop, 64, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->d_stop, c->h_stop, 0) != cudaSuccess ||
        cudaEventCreate(&c->ev_k0) != cudaSuccess || cudaEventCreate(&c->ev_k1) != cudaSuccess) {
        tg_ctx_destroy(c);
        return TG_ERR_CUDA;
    }
    *(volatile u32 *)c->h_cancel = 0;
    memset(c->h_status, 0, kMaxGraphs * sizeof(i32));
    if (cudaMemsetAsync(c->ctl, 0, sizeof(LaunchCtl), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->descs, 0, (size_t)kMaxGraphs * sizeof(GDesc), c->stream) != cudaSuccess) {
        tg_ctx_destroy(c);
        return TG_ERR_CUDA;
    }
    c->dirty = true;
    if (clear_if_dirty(c) != TG_OK || cudaStreamSynchronize(c->stream) != cudaSuccess) {
        tg_ctx_destroy(c);
        return TG_ERR_CUDA;
    }
    *out = c;
    return TG_OK;
}

int tg_serve_stop(tg_ctx *c);

int tg_ctx_destroy(tg_ctx *c)
{
    if (!c)
        return TG_ERR_INVALID;
    if (c->serving)
        tg_serve_stop(c);   // a resident scheduler would otherwise run to its time limit
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->subs)
        if (kv.second.ev)
            cudaEventDestroy(kv.second.ev);
    if (c->h_cancel)
        cudaFreeHost(c->h_cancel);
    if (c->h_status)
        cudaFreeHost(c->h_status);
    if (c->h_stage)
        cudaFreeHost(c->h_stage);
    if (c->h_sub)
        cudaFreeHost(c->h_sub);
    if (c->h_comp)
        cudaFreeHost(c->h_comp);
    if (c->h_stop)
        cudaFreeHost(c->h_stop);
    delete[] c->by_gid;
    if (c->capture_stream)
        cudaStreamDestroy(c->capture_stream);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->pk_scratch)
        cudaFree(c->pk_scratch);
    if (c->d_rb)
        cudaFree(c->d_rb);
    if (c->h_pkflags)
        cudaFreeHost(c->h_pkflags);
    for (cudaEvent_t ev : c->pk_ev)
        if (ev)
            cudaEventDestroy(ev);
    if (c->ev_k0)
        cudaEventDestroy(c->ev_k0);
    if (c->ev_k1)
        cudaEventDestroy(c->ev_k1);
    // batches and graphs the caller did not destroy (their device memory is
    // the caller's arena; only host objects, captured graphs and events)
    for (tg_batch *b : c->live_batches) {
        if (b->exec)
            cudaGraphExecDestroy(b->exec);
        if (b->done)
            cudaEventDestroy(b->done);
        delete b;
    }
    for (tg_graph *g : c->live_graphs) {
        if (g->cap_exec)
            cudaGraphExecDestroy(g->cap_exec);
        if (g->ready)
            cudaEventDestroy(g->ready);
        delete g;
    }
    delete c;
    return TG_OK;
}

int tg_ctx_set_launch(tg_ctx *c, const tg_ctx_opts *launch)
{
    if (!c || !launch)
        return TG_ERR_INVALID;
    Geometry g;
    int rc = resolve_geometry(c, *launch, g);
    if (rc != TG_OK)
        return rc;
    c->geo = g;
    geometry_to_opts(g, c->opts);
    return TG_OK;
}

int tg_ctx_get_opts(const tg_ctx *c, tg_ctx_opts *o)
{
    if (!c || !o)
        return TG_ERR_INVALID;
    *o = c->opts;
    o->max_nodes = c->node_cap;
    o->max_edges = c->edge_cap;
    o->mem_budget_bytes = c->budget;
    return TG_OK;
}

static bool is_cond(u32 kind) { return kind >= TG_COND_BRANCH && kind <= TG_COND_CONST; }

// Pool space of a new graph: a chunk-aligned execution range, and in the
// edge pool its successor lists (a module task's list led by the slot id of
// the graph it composes) and its sources; a graph slot; the budget.
static int graph_alloc(tg_ctx *c, u32 n, u32 m, u32 n_mod, u32 n_src, u32 n_cond, u32 seed, tg_graph **out)
{
    const u64 n_chunks = ((u64)n + kChunk - 1) >> kChunkShift;
    const u64 bytes = n_chunks * kChunk * 36 + ((u64)m + n_mod + n_src) * 4;
    if (c->used + bytes > c->budget || c->free_gids.empty())
        return TG_ERR_BUDGET;
    tg_graph *g = new (std::nothrow) tg_graph();
    if (!g)
        return TG_ERR_INVALID;
    if (!c->nodes.alloc(n_chunks, g->chunk_off)) {
        delete g;
        return TG_ERR_BUDGET;
    }
    c->live_graphs.insert(g);
    g->n_chunks = n_chunks;
    g->node_off = g->chunk_off << kChunkShift;
    g->edge_len = (u64)m + n_mod + n_src;
    if (!c->edge_pool.alloc(g->edge_len, g->edge_off)) {
        c->nodes.release(g->chunk_off, n_chunks);
        c->live_graphs.erase(g);
        delete g;
        return TG_ERR_BUDGET;
    }
    g->gid = c->free_gids.back();
    c->free_gids.pop_back();
    c->used += bytes;
    g->ctx = c;
    g->n = n;
    g->m = m;
    g->n_src = n_src;
    g->n_cond = n_cond;
    g->n_mod = n_mod;
    g->seed = seed;
    g->bytes = bytes;
    *out = g;
    return TG_OK;
}

static int graph_create(tg_ctx *c, uint32_t n, const uint8_t *kinds, const uint32_t *params, uint32_t m,
                        const uint32_t *src, const uint32_t *dst, const uint8_t *weak, uint32_t seed,
                        tg_graph *const *modules, tg_graph **out)
{
    if (!c || !out || n == 0 || !kinds || !params || (m && (!src || !dst)))
        return TG_ERR_INVALID;
    *out = nullptr;
    const u64 t0 = now_ns();
    // ---- validation (same order as the rule statement in tg.h)
    u32 n_cond = 0, n_mod = 0;
    for (u32 v = 0; v < n; ++v) {
        if (kinds[v] > TG_SUBFLOW || (kinds[v] >= TG_MODULE && !modules))
            return TG_ERR_INVALID;
        if (kinds[v] == TG_COND_LOOP && ((params[v] >> 16) & 0xFFu) == 0u)
            return TG_ERR_INVALID;
        if (modules) {
            const tg_graph *mg = modules[v];
            if ((kinds[v] >= TG_MODULE) != (mg != nullptr))
                return TG_ERR_INVALID;
            if (mg && (mg->ctx != c || mg->tmpl != nullptr))
                return TG_ERR_INVALID;
            if (mg && kinds[v] == TG_SUBFLOW && mg->n_mod != 0)
                return TG_ERR_INVALID;   // a template holds no module or subflow tasks
        }
        n_cond += is_cond(kinds[v]);
        n_mod += kinds[v] >= TG_MODULE;
    }
    // degrees, with each edge's endpoints checked before they are used
    std::vector<u32> outdeg(n, 0), sin(n, 0), win(n, 0);
    for (u32 e = 0; e < m; ++e) {
        const u32 sv = src[e], dv = dst[e];
        if (sv >= n || dv >= n)
            return TG_ERR_INVALID;
        outdeg[sv]++;
        if (!is_cond(kinds[sv]))
            sin[dv]++;
        else
            win[dv]++;
    }
    u32 n_src = 0;
    for (u32 v = 0; v < n; ++v) {
        if (is_cond(kinds[v]) && outdeg[v] == 0)
            return TG_ERR_INVALID;
        if (outdeg[v] > kMaxDegree || sin[v] > kMaxDegree)
            return TG_ERR_INVALID;
        n_src += (sin[v] == 0 && win[v] == 0);
    }
    if (weak)
        for (u32 e = 0; e < m; ++e)
            if ((weak[e] != 0) != is_cond(kinds[src[e]]))
                return TG_ERR_EDGE_KIND;
    if (n_src == 0)
        return TG_ERR_NO_SOURCE;

    tg_graph *g = nullptr;
    if (int ra = graph_alloc(c, n, m, n_mod, n_src, n_cond, seed, &g); ra != TG_OK)
        return ra;
    const u64 n_chunks = g->n_chunks;

    // ---- pack: successors in insertion order (graph-local ids), sources,
    // then the 32-byte task records (W = strong in-degree, cnt = dig = 0)
    const size_t edge_bytes = (size_t)g->edge_len * 4;
    const size_t chunk_bytes = (size_t)n_chunks * 4;
    // staging: successor lists, chunk table, descriptor, then the records on
    // a 256-byte boundary
    const size_t rec_at = ((g->edge_off & 63u) * 4u + edge_bytes + chunk_bytes + sizeof(GDesc) + 255) & ~(size_t)255;
    int rc = ensure_stage(c, rec_at + (size_t)n * sizeof(NodeSlot));
    if (rc != TG_OK) {
        tg_graph_destroy(c, g);
        return rc;
    }
    if (modules)
        for (u32 v = 0; v < n; ++v)
            if (kinds[v] == TG_SUBFLOW) {
                tg_graph *inst = nullptr;
                int ri = tg_instance_create(c, modules[v], &inst);
                if (ri != TG_OK) {
                    tg_graph_destroy(c, g);
                    return ri;
                }
                g->sub_insts.push_back(inst);
            }
    cudaStreamSynchronize(c->side);   // the staging buffer may still feed an earlier upload
    // the staged successor lists start at the same offset within 256 bytes
    // as their device copy
    char *stage = c->h_stage + (g->edge_off & 63u) * 4u;
    u32 *he = (u32 *)stage;
    NodeSlot *hs = (NodeSlot *)(c->h_stage + rec_at);
    u32 *hc = (u32 *)(stage + edge_bytes);
    const bool stream_records = ((uintptr_t)hs & 15u) == 0u;
    const u32 edge_base = (u32)g->edge_off;
    u32 acc = 0, sub_i = 0;
    for (u32 v = 0; v < n; ++v) {
        NodeSlot s;
        const u32 kind = kinds[v];
        u32 arg = 0;
        if (kind == TG_COND_LOOP)
            arg = (params[v] >> 16) & 0xFFu;
        else if (kind == TG_COND_CONST || kind == TG_SUBFLOW)
            arg = params[v] >> 24;   // the constant; a subflow's detach bit
        s.succ_off = edge_base + acc;
        s.deg = outdeg[v] | (sin[v] << 16);
        s.prm = (params[v] & 0xFFFFu) | (kind << 16) | (arg << 24);
        s.lid = v;
        s.W = sin[v];
        s.cnt = 0;
        s.dig = 0;
#if defined(__x86_64__)
        // only the copy engine reads the staging buffer: streaming stores
        // skip the cache (three times faster for a large graph)
        if (stream_records) {
            _mm_stream_si128(reinterpret_cast<__m128i *>(&hs[v]),
                             _mm_setr_epi32((int)s.succ_off, (int)s.deg, (int)s.prm, (int)s.lid));
            _mm_stream_si128(reinterpret_cast<__m128i *>(&hs[v]) + 1, _mm_setr_epi32((int)sin[v], 0, 0, 0));
        } else {
            memcpy(&hs[v], &s, sizeof(s));
        }
#else
        (void)stream_records;
        memcpy(&hs[v], &s, sizeof(s));
#endif
        if (kind == TG_MODULE)
            he[acc++] = modules[v]->gid;
        else if (kind == TG_SUBFLOW)
            he[acc++] = g->sub_insts[sub_i++]->gid;
        outdeg[v] = acc;   // reuse as the fill cursor
        acc += (u32)(s.deg & 0xFFFFu);
    }
    // a strong edge to a task with no other strong in-edge is marked: its
    // release needs no join-word update
    for (u32 e = 0; e < m; ++e)
        he[outdeg[src[e]]++] = dst[e] | ((!is_cond(kinds[src[e]]) && sin[dst[e]] == 1u) ? kSoleBit : 0u);
    for (u32 v = 0, k = 0; v < n; ++v)
        if (sin[v] == 0 && win[v] == 0)
            he[m + n_mod + k++] = v;
    if (modules)
        for (u32 v = 0; v < n; ++v)
            if (kinds[v] == TG_MODULE && std::find(g->mods.begin(), g->mods.end(), modules[v]) == g->mods.end()) {
                g->mods.push_back(modules[v]);
                modules[v]->n_refs++;
            }
    for (u64 k = 0; k < n_chunks; ++k)
        hc[k] = g->gid;
    const u64 t1 = now_ns();

    GDesc d{};
    d.pe = 0;
    d.status = 0;
    d.seed = seed;
    d.node_off = (u32)g->node_off;
    d.n = n;
    d.src_off = edge_base + m + n_mod;
    d.ret = kEmpty32;
    d.n_src = n_src;
    d.exec_cap = (u32)std::min<u64>(c->opts.exec_cap, 0xFFFFFFFFull);
#if defined(__x86_64__)
    _mm_sfence();   // the streamed records are in memory before the copy engine reads them
#endif
    memcpy(stage + edge_bytes + chunk_bytes, &d, sizeof(d));
    // The upload goes on the side stream: the new graph's slot and node and
    // edge ranges are in no running launch's use (a destroyed graph's ranges
    // are freed only after its last launch ended), so a graph can be
    // ingested while another one runs on the context stream.  The call
    // returns once the upload is complete.
    cudaError_t e1 = cudaMemcpyAsync(c->edges + g->edge_off, he, edge_bytes, cudaMemcpyHostToDevice, c->side);
    cudaError_t e2 = cudaMemcpyAsync(c->slots + g->node_off, hs, (size_t)n * sizeof(NodeSlot),
                                     cudaMemcpyHostToDevice, c->side);
    cudaError_t e3 = cudaMemcpyAsync(c->chunk_gid + g->chunk_off, hc, chunk_bytes, cudaMemcpyHostToDevice, c->side);
    cudaError_t e4 = cudaMemcpyAsync(c->descs + g->gid, stage + edge_bytes + chunk_bytes, sizeof(GDesc),
                                     cudaMemcpyHostToDevice, c->side);
    cudaError_t e5 = cudaStreamSynchronize(c->side);
    if (e1 || e2 || e3 || e4 || e5) {
        tg_graph_destroy(c, g);
        return TG_ERR_CUDA;
    }
    g->pack_ns = t1 - t0;
    g->upload_ns = now_ns() - t1;
    *out = g;
    return TG_OK;
}

int tg_graph_create(tg_ctx *c, uint32_t n, const uint8_t *kinds, const uint32_t *params, uint32_t m,
                    const uint32_t *src, const uint32_t *dst, const uint8_t *weak, uint32_t seed, tg_graph **out)
{
    return graph_create(c, n, kinds, params, m, src, dst, weak, seed, nullptr, out);
}

int tg_graph_create_dev(tg_ctx *c, uint32_t n, const uint8_t *kinds, const uint32_t *params, uint32_t m,
                        const uint32_t *src, const uint32_t *dst, const uint8_t *weak, uint32_t seed, tg_graph **out)
{
    if (!c || !out || n == 0 || !kinds || !params || (m && (!src || !dst)))
        return TG_ERR_INVALID;
    *out = nullptr;
    // scratch for the copied inputs, the counts and the sort; an earlier
    // call has finished with it (each call ends synchronised)
    const size_t need = pack_scratch_bytes(n, m);
    if (c->pk_bytes < need) {
        if (c->pk_scratch) {
            cudaFree(c->pk_scratch);
            c->pk_scratch = nullptr;
            c->pk_bytes = 0;
        }
        if (cudaMalloc((void **)&c->pk_scratch, need) != cudaSuccess) {
            (void)cudaGetLastError();
            return TG_ERR_BUDGET;
        }
        c->pk_bytes = need;
    }
    if (!c->h_pkflags) {
        TG_CUDA(cudaHostAlloc((void **)&c->h_pkflags, 256, cudaHostAllocDefault));
        for (cudaEvent_t &ev : c->pk_ev)
            TG_CUDA(cudaEventCreate(&ev));
    }
    PackBufs b;
    pack_carve(c->pk_scratch, n, m, b);
    cudaStream_t st = c->side;
    TG_CUDA(cudaEventRecord(c->pk_ev[0], st));
    TG_CUDA(cudaMemcpyAsync(b.kinds, kinds, n, cudaMemcpyHostToDevice, st));
    TG_CUDA(cudaMemcpyAsync(b.params, params, (size_t)4 * n, cudaMemcpyHostToDevice, st));
    if (m) {
        TG_CUDA(cudaMemcpyAsync(b.src, src, (size_t)4 * m, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(b.dst, dst, (size_t)4 * m, cudaMemcpyHostToDevice, st));
        if (weak)
            TG_CUDA(cudaMemcpyAsync(b.weak, weak, m, cudaMemcpyHostToDevice, st));
    }
    TG_CUDA(cudaEventRecord(c->pk_ev[1], st));
    TG_CUDA(pack_validate(b, n, m, weak != nullptr, st));
    TG_CUDA(cudaMemcpyAsync(c->h_pkflags, b.flags, PK_FLAGS * sizeof(u32), cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    // the host packer's order of statuses
    const u32 *f = c->h_pkflags;
    if (f[PK_INVALID])
        return TG_ERR_INVALID;
    if (f[PK_EDGE_KIND])
        return TG_ERR_EDGE_KIND;
    if (f[PK_NSRC] == 0u)
        return TG_ERR_NO_SOURCE;
    tg_graph *g = nullptr;
    if (int ra = graph_alloc(c, n, m, 0u, f[PK_NSRC], f[PK_NCOND], seed, &g); ra != TG_OK)
        return ra;
    PackDest d{};
    d.slots = c->slots + g->node_off;
    d.edges = c->edges + g->edge_off;
    d.edge_base = (u32)g->edge_off;
    d.chunk_gid = c->chunk_gid + g->chunk_off;
    d.n_chunks = (u32)g->n_chunks;
    d.gid = g->gid;
    d.desc = c->descs + g->gid;
    d.seed = seed;
    d.node_off = (u32)g->node_off;
    d.n_src = g->n_src;
    d.exec_cap = (u32)std::min<u64>(c->opts.exec_cap, 0xFFFFFFFFull);
    cudaError_t e = pack_build(b, n, m, d, st);
    if (e == cudaSuccess)
        e = cudaEventRecord(c->pk_ev[2], st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        tg_graph_destroy(c, g);
        return TG_ERR_CUDA;
    }
    float up = 0.f, pk = 0.f;
    if (cudaEventElapsedTime(&up, c->pk_ev[0], c->pk_ev[1]) == cudaSuccess)
        g->upload_ns = (u64)((double)up * 1e6);
    if (cudaEventElapsedTime(&pk, c->pk_ev[1], c->pk_ev[2]) == cudaSuccess)
        g->pack_ns = (u64)((double)pk * 1e6);
    *out = g;
    return TG_OK;
}

int tg_graph_create_composed(tg_ctx *c, uint32_t n, const uint8_t *kinds, const uint32_t *params, uint32_t m,
                             const uint32_t *src, const uint32_t *dst, const uint8_t *weak, uint32_t seed,
                             tg_graph *const *modules, tg_graph **out)
{
    if (!modules)
        return TG_ERR_INVALID;
    return graph_create(c, n, kinds, params, m, src, dst, weak, seed, modules, out);
}

}  // extern "C"

// Write an instance's records (re-armed from the template's records), chunk
// table and descriptor on the side stream; later launches wait for `ready`.
static int instance_setup(tg_ctx *c, tg_graph *g)
{
    tg_graph *src = g->tmpl ? g->tmpl : g;
    std::vector<u32> hc(g->n_chunks, g->gid);
    GDesc d{};
    d.seed = g->seed;
    d.node_off = (u32)g->node_off;
    d.n = g->n;
    d.src_off = (u32)(src->edge_off + src->m);
    d.n_src = g->n_src;
    d.exec_cap = (u32)std::min<u64>(c->opts.exec_cap, 0xFFFFFFFFull);
    TG_CUDA(launch_instance_rearm(c->slots, src->node_off, g->node_off, g->n, c->side));
    TG_CUDA(cudaMemcpyAsync(c->chunk_gid + g->chunk_off, hc.data(), hc.size() * 4, cudaMemcpyHostToDevice, c->side));
    TG_CUDA(cudaMemcpyAsync(c->descs + g->gid, &d, sizeof(d), cudaMemcpyHostToDevice, c->side));
    if (!g->ready)
        TG_CUDA(cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming));
    TG_CUDA(cudaEventRecord(g->ready, c->side));
    g->setup_pending = false;
    return TG_OK;
}

extern "C" {

int tg_instance_create(tg_ctx *c, tg_graph *t, tg_graph **out)
{
    if (!c || !t || !out || t->ctx != c || t->n_mod)
        return TG_ERR_INVALID;
    *out = nullptr;
    tg_graph *src = t->tmpl ? t->tmpl : t;
    const u64 bytes = src->n_chunks * kChunk * 36;
    if (c->used + bytes > c->budget || c->free_gids.empty())
        return TG_ERR_BUDGET;
    u64 chunk_off = 0;
    if (!c->nodes.alloc(src->n_chunks, chunk_off))
        return TG_ERR_BUDGET;
    tg_graph *g = new (std::nothrow) tg_graph();
    if (!g) {
        c->nodes.release(chunk_off, src->n_chunks);
        return TG_ERR_INVALID;
    }
    *g = *src;
    c->live_graphs.insert(g);
    g->chunk_off = chunk_off;
    g->tmpl = src;
    g->n_inst = 0;
    g->busy = nullptr;
    g->ready = nullptr;
    // what belongs to the template alone stays with it
    g->n_refs = 0;
    g->n_batches = 0;
    g->mods.clear();
    g->sub_insts.clear();
    g->cap_exec = nullptr;
    g->cap_streams = 0;
    g->serve_ticket = 0;
    g->setup_pending = false;
    g->node_off = g->chunk_off << kChunkShift;
    g->edge_len = 0;   // the packed form stays with the template
    g->bytes = bytes;
    g->pack_ns = 0;
    g->gid = c->free_gids.back();
    c->free_gids.pop_back();
    c->used += bytes;
    src->n_inst++;
    if (c->serving) {
        // the resident scheduler writes the descriptor and chunk table when
        // it claims the instance's first submission
        g->setup_pending = true;
        *out = g;
        return TG_OK;
    }
    const u64 t0 = now_ns();
    int rc = instance_setup(c, g);
    if (rc != TG_OK) {
        tg_graph_destroy(c, g);
        return rc;
    }
    g->upload_ns = now_ns() - t0;
    *out = g;
    return TG_OK;
}

int tg_graph_destroy(tg_ctx *c, tg_graph *g)
{
    if (!c || !g || g->ctx != c)
        return TG_ERR_INVALID;
    if (g->n_inst > 0 || g->serve_ticket != 0 || g->n_refs > 0 || g->n_batches > 0)
        return TG_ERR_BUSY;   // instances use its packed form, or it is served, composed or in a batch
    if (g->busy)
        cudaEventSynchronize(g->busy);
    if (g->ready) {
        cudaEventSynchronize(g->ready);
        cudaEventDestroy(g->ready);
    }
    if (g->cap_exec)
        cudaGraphExecDestroy(g->cap_exec);
    for (tg_graph *mg : g->mods)
        mg->n_refs--;
    for (tg_graph *inst : g->sub_insts)
        tg_graph_destroy(c, inst);
    g->sub_insts.clear();
    c->nodes.release(g->chunk_off, g->n_chunks);
    if (g->edge_len)
        c->edge_pool.release(g->edge_off, g->edge_len);
    if (g->tmpl)
        g->tmpl->n_inst--;
    c->free_gids.push_back(g->gid);
    c->used -= g->bytes;
    for (auto it = c->subs.begin(); it != c->subs.end();) {
        if (it->second.g == g) {
            if (it->second.ev)
                cudaEventDestroy(it->second.ev);
            it = c->subs.erase(it);
        } else {
            ++it;
        }
    }
    c->live_graphs.erase(g);
    delete g;
    return TG_OK;
}

int tg_graph_get_info(const tg_graph *g, tg_graph_info *info)
{
    if (!g || !info)
        return TG_ERR_INVALID;
    info->n_nodes = g->n;
    info->n_edges = g->m;
    info->n_sources = g->n_src;
    info->n_conditions = g->n_cond;
    info->device_bytes = g->bytes;
    info->pack_ns = g->pack_ns;
    info->upload_ns = g->upload_ns;
    return TG_OK;
}

static int serve_submit(tg_ctx *c, tg_graph *g, uint64_t *ticket);
static int finish_sub(tg_ctx *c, Submission &s);

// Every graph that the module and subflow tasks of `roots` reach
// (transitively), the roots themselves excluded.
static std::vector<tg_graph *> composition_closure(const std::vector<tg_graph *> &roots)
{
    std::vector<tg_graph *> todo, seen;
    for (tg_graph *r : roots) {
        todo.insert(todo.end(), r->mods.begin(), r->mods.end());
        todo.insert(todo.end(), r->sub_insts.begin(), r->sub_insts.end());
    }
    while (!todo.empty()) {
        tg_graph *mg = todo.back();
        todo.pop_back();
        if (std::find(roots.begin(), roots.end(), mg) != roots.end() ||
            std::find(seen.begin(), seen.end(), mg) != seen.end())
            continue;
        seen.push_back(mg);
        todo.insert(todo.end(), mg->mods.begin(), mg->mods.end());
        todo.insert(todo.end(), mg->sub_insts.begin(), mg->sub_insts.end());
    }
    return seen;
}

int tg_submit(tg_ctx *c, tg_graph *g, uint64_t *ticket)
{
    if (!c || !g || g->ctx != c || !ticket)
        return TG_ERR_INVALID;
    if (c->serving)
        return g->n_mod ? TG_ERR_INVALID : serve_submit(c, g, ticket);
    if (graph_busy(g))
        return TG_ERR_BUSY;
    // the graph's earlier submissions have finished: take their statuses (a
    // failed run marks the queues for clearing) and release their tickets
    for (auto it = c->subs.begin(); it != c->subs.end();) {
        if (it->second.g == g) {
            finish_sub(c, it->second);
            if (it->second.ev)
                cudaEventDestroy(it->second.ev);
            it = c->subs.erase(it);
        } else {
            ++it;
        }
    }
    int rc = clear_if_dirty(c);
    if (rc != TG_OK)
        return rc;
    if (g->setup_pending) {
        int rc2 = instance_setup(c, g);
        if (rc2 != TG_OK)
            return rc2;
    }
    if (g->ready)
        TG_CUDA(cudaStreamWaitEvent(c->stream, g->ready, 0));
    // the graph's own tuned geometry, else the context's
    const Geometry &geo = g->has_geo ? g->geo : c->geo;
    KParams p = base_params(c, geo);
    p.lt = nullptr;
    p.n_graphs = 1;
    p.single_gid = g->gid;
    p.max_n = g->n;
    p.total_sources = g->n_src;
    if (g->n_cond == 0 && g->n_mod == 0)
        p.flags |= kFlagAcyclic;
    if (g->n_mod) {
        // every graph the composition reaches starts idle from its initial state
        p.has_modules = 1u;
        for (tg_graph *mg : composition_closure({g})) {
            if (mg->ready)
                TG_CUDA(cudaStreamWaitEvent(c->stream, mg->ready, 0));
            TG_CUDA(launch_module_rearm(p, mg->gid, mg->n, c->stream));
        }
    }
    Submission s;
    s.g = g;
    TG_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
    TG_CUDA(launch_rearm(p, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(launch_sched(p, geo.blocks, geo.threads, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    TG_CUDA(launch_finalize(p, c->stream));
    TG_CUDA(cudaEventRecord(s.ev, c->stream));
    c->last_geo = geo;
    c->timed = true;
    g->busy = s.ev;
    *ticket = c->next_ticket++;
    c->subs[*ticket] = s;
    return TG_OK;
}

static int finish_sub(tg_ctx *c, Submission &s)
{
    if (s.status == TG_PENDING) {
        s.status = c->h_status[s.g->gid];
        note_status(c, s.status);
        if (s.g->busy == s.ev)
            s.g->busy = nullptr;
    }
    return s.status;
}

static int serve_poll(tg_ctx *c, uint64_t ticket);

int tg_poll(tg_ctx *c, uint64_t ticket)
{
    if (!c)
        return TG_ERR_INVALID;
    if (c->serving || c->serve_done.count(ticket))
        return serve_poll(c, ticket);
    auto it = c->subs.find(ticket);
    if (it == c->subs.end())
        return TG_ERR_INVALID;
    Submission &s = it->second;
    if (s.status != TG_PENDING)
        return s.status;
    cudaError_t q = cudaEventQuery(s.ev);
    if (q == cudaErrorNotReady)
        return TG_PENDING;
    if (q != cudaSuccess)
        return TG_ERR_CUDA;
    return finish_sub(c, s);
}

int tg_wait(tg_ctx *c, uint64_t ticket)
{
    if (!c)
        return TG_ERR_INVALID;
    if (c->serving || c->serve_done.count(ticket)) {
        for (;;) {
            int st = serve_poll(c, ticket);
            if (st != TG_PENDING)
                return st;
            if (cudaStreamQuery(c->stream) != cudaErrorNotReady)
                return serve_poll(c, ticket);   // the server ended
        }
    }
    auto it = c->subs.find(ticket);
    if (it == c->subs.end())
        return TG_ERR_INVALID;
    Submission &s = it->second;
    if (s.status != TG_PENDING)
        return s.status;
    if (cudaEventSynchronize(s.ev) != cudaSuccess)
        return TG_ERR_CUDA;
    return finish_sub(c, s);
}

int tg_run(tg_ctx *c, tg_graph *g)
{
    if (c && c->serving)
        return TG_ERR_BUSY;
    uint64_t t = 0;
    int rc = tg_submit(c, g, &t);
    if (rc != TG_OK)
        return rc;
    rc = tg_wait(c, t);
    auto it = c->subs.find(t);
    if (it != c->subs.end()) {
        cudaEventDestroy(it->second.ev);
        c->subs.erase(it);
    }
    return rc;
}

int tg_cancel(tg_ctx *c)
{
    if (!c)
        return TG_ERR_INVALID;
    *(volatile u32 *)c->h_cancel = 1u;
    return TG_OK;
}

int tg_result_copy(tg_ctx *c, const tg_graph *g, uint32_t *out, uint32_t *cnt, uint32_t *dig,
                   uint64_t *total_execs)
{
    if (!c || !g || g->ctx != c)
        return TG_ERR_INVALID;
    if (!c->serving) {
        // After the graph's own last launch -- not the whole context stream,
        // where a graph submitted later may run meanwhile -- the counts and
        // digests are packed on the device (8 bytes per task instead of the
        // 32-byte record) into a read-back buffer of the context, and both
        // arrays come back through the pinned staging buffer, all on the
        // side stream.
        const size_t out_bytes = (size_t)g->n * 4, word_bytes = (size_t)g->n * 8;
        int rs = ensure_stage(c, out_bytes + word_bytes);
        if (rs != TG_OK)
            return rs;
        if (c->rb_bytes < word_bytes) {
            TG_CUDA(cudaStreamSynchronize(c->side));
            if (c->d_rb)
                cudaFree(c->d_rb);
            c->d_rb = nullptr;
            c->rb_bytes = 0;
            if (cudaMalloc((void **)&c->d_rb, word_bytes) != cudaSuccess) {
                (void)cudaGetLastError();
                return TG_ERR_BUDGET;
            }
            c->rb_bytes = word_bytes;
        }
        if (g->busy)
            TG_CUDA(cudaStreamWaitEvent(c->side, g->busy, 0));
        else if (g->n_refs || g->tmpl)
            TG_CUDA(cudaStreamSynchronize(c->stream));   // it may run inside the launch of a graph composing it
        TG_CUDA(launch_result_gather(c->slots, (u32)g->node_off, g->n, c->d_rb, c->side));
        TG_CUDA(cudaMemcpyAsync(c->h_stage, c->d_rb, word_bytes, cudaMemcpyDeviceToHost, c->side));
        TG_CUDA(cudaMemcpyAsync(c->h_stage + word_bytes, c->outv + g->node_off, out_bytes, cudaMemcpyDeviceToHost,
                                c->side));
        TG_CUDA(cudaStreamSynchronize(c->side));
        const u64 *hw = (const u64 *)c->h_stage;
        const u32 *ho = (const u32 *)(c->h_stage + word_bytes);
        u64 tot = 0;
        for (u32 v = 0; v < g->n; ++v) {
            const u32 k = (u32)hw[v];
            if (cnt)
                cnt[v] = k;
            if (dig)
                dig[v] = (u32)(hw[v] >> 32);
            if (out)
                out[v] = k == 0 ? 0u : ho[v];   // never executed: 0 (an instance's range is not zeroed)
            tot += k;
        }
        if (total_execs)
            *total_execs = tot;
        return TG_OK;
    }
    if (out)
        TG_CUDA(cudaMemcpyAsync(out, c->outv + g->node_off, (size_t)g->n * 4, cudaMemcpyDeviceToHost, c->side));
    TG_CUDA(cudaStreamSynchronize(c->side));
    if (out || cnt || dig || total_execs) {
        std::vector<NodeSlot> tmp(g->n);
        TG_CUDA(cudaMemcpyAsync(tmp.data(), c->slots + g->node_off, (size_t)g->n * sizeof(NodeSlot),
                                cudaMemcpyDeviceToHost, c->side));
        TG_CUDA(cudaStreamSynchronize(c->side));
        u64 tot = 0;
        for (u32 v = 0; v < g->n; ++v) {
            const u32 k = tmp[v].cnt & ~(kInflight | kAwait);
            if (cnt)
                cnt[v] = k;
            if (dig)
                dig[v] = tmp[v].dig;
            if (out && k == 0)
                out[v] = 0;   // never executed (an instance's range is not zeroed)
            tot += k;
        }
        if (total_execs)
            *total_execs = tot;
    }
    return TG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// capturer baseline (Algorithm 1): levelize, round-robin streams, capture
// ---------------------------------------------------------------------------
namespace {

// Longest-path levels of a DAG given as successor lists; index = position in
// the level by ascending id.  False on a cycle.
bool levelize_csr(u32 n, const std::vector<u32> &off, const std::vector<u32> &adj, std::vector<u32> &level,
                  std::vector<u32> &index, u32 &n_levels)
{
    std::vector<u32> indeg(n, 0);
    for (u32 e = 0; e < off[n]; ++e)
        indeg[adj[e]]++;
    level.assign(n, 0);
    std::vector<u32> order;
    order.reserve(n);
    for (u32 v = 0; v < n; ++v)
        if (indeg[v] == 0)
            order.push_back(v);
    for (size_t h = 0; h < order.size(); ++h) {
        const u32 v = order[h];
        for (u32 e = off[v]; e < off[v + 1]; ++e) {
            const u32 t = adj[e];
            level[t] = std::max(level[t], level[v] + 1u);
            if (--indeg[t] == 0)
                order.push_back(t);
        }
    }
    if (order.size() != n)
        return false;
    n_levels = 0;
    for (u32 v = 0; v < n; ++v)
        n_levels = std::max(n_levels, level[v] + 1u);
    std::vector<u32> fill(n_levels, 0);
    index.assign(n, 0);
    for (u32 v = 0; v < n; ++v)   // ascending id within each level
        index[v] = fill[level[v]]++;
    return true;
}

bool csr_from_edges(u32 n, u32 m, const u32 *src, const u32 *dst, std::vector<u32> &off, std::vector<u32> &adj)
{
    off.assign(n + 1, 0);
    for (u32 e = 0; e < m; ++e) {
        if (src[e] >= n || dst[e] >= n)
            return false;
        off[src[e] + 1]++;
    }
    for (u32 v = 0; v < n; ++v)
        off[v + 1] += off[v];
    adj.assign(m, 0);
    std::vector<u32> cur(off.begin(), off.end() - 1);
    for (u32 e = 0; e < m; ++e)
        adj[cur[src[e]]++] = dst[e];
    return true;
}

}  // namespace

extern "C" {

int tg_levelize(uint32_t n, uint32_t m, const uint32_t *src, const uint32_t *dst, uint32_t *level,
                uint32_t *index, uint32_t *n_levels)
{
    if (n == 0 || !level || !index || (m && (!src || !dst)))
        return TG_ERR_INVALID;
    std::vector<u32> off, adj, lv, ix;
    u32 nl = 0;
    if (!csr_from_edges(n, m, src, dst, off, adj) || !levelize_csr(n, off, adj, lv, ix, nl))
        return TG_ERR_INVALID;
    std::copy(lv.begin(), lv.end(), level);
    std::copy(ix.begin(), ix.end(), index);
    if (n_levels)
        *n_levels = nl;
    return TG_OK;
}

int tg_stream_plan(uint32_t n, uint32_t m, const uint32_t *src, const uint32_t *dst, uint32_t max_streams,
                   uint32_t *stream, uint32_t *n_events, uint32_t *n_waits)
{
    if (n == 0 || !stream || max_streams == 0 || max_streams > 32 || (m && (!src || !dst)))
        return TG_ERR_INVALID;
    std::vector<u32> off, adj, lv, ix;
    u32 nl = 0;
    if (!csr_from_edges(n, m, src, dst, off, adj) || !levelize_csr(n, off, adj, lv, ix, nl))
        return TG_ERR_INVALID;
    for (u32 v = 0; v < n; ++v)
        stream[v] = ix[v] % max_streams;
    u32 events = 0;
    std::vector<std::pair<u32, u32>> cross;
    for (u32 v = 0; v < n; ++v) {
        bool rec = false;
        for (u32 e = off[v]; e < off[v + 1]; ++e)
            if (stream[adj[e]] != stream[v]) {
                rec = true;
                cross.emplace_back(v, adj[e]);
            }
        events += rec;
    }
    std::sort(cross.begin(), cross.end());
    cross.erase(std::unique(cross.begin(), cross.end()), cross.end());
    if (n_events)
        *n_events = events;
    if (n_waits)
        *n_waits = (u32)cross.size();
    return TG_OK;
}

int tg_graph_packed_copy(tg_ctx *c, const tg_graph *g, uint32_t *records, uint32_t *edges, uint64_t *edge_words)
{
    if (!c || !g || g->ctx != c)
        return TG_ERR_INVALID;
    const tg_graph *t = g->tmpl ? g->tmpl : g;   // an instance shares its template's lists
    if (edge_words)
        *edge_words = t->edge_len;
    if (!c->serving)
        TG_CUDA(cudaStreamSynchronize(c->stream));
    if (records) {
        TG_CUDA(cudaMemcpy(records, c->slots + g->node_off, (size_t)g->n * sizeof(NodeSlot), cudaMemcpyDeviceToHost));
        for (u32 v = 0; v < g->n; ++v)
            records[8ull * v] -= (u32)t->edge_off;
    }
    if (edges && t->edge_len)
        TG_CUDA(cudaMemcpy(edges, c->edges + t->edge_off, (size_t)t->edge_len * 4, cudaMemcpyDeviceToHost));
    return TG_OK;
}

int tg_graph_dot(tg_ctx *c, const tg_graph *g, char *buf, size_t cap, size_t *len)
{
    if (!c || !g || g->ctx != c || !len)
        return TG_ERR_INVALID;
    const tg_graph *t = g->tmpl ? g->tmpl : g;
    // (the immutable half of the template's own records: successor range,
    // degrees, kind and parameters)
    std::vector<NodeSlot> rec(g->n);
    std::vector<u32> ed(t->edge_len);
    if (!c->serving)
        TG_CUDA(cudaStreamSynchronize(c->stream));
    TG_CUDA(cudaMemcpy(rec.data(), c->slots + t->node_off, (size_t)g->n * sizeof(NodeSlot),
                       cudaMemcpyDeviceToHost));
    if (!ed.empty())
        TG_CUDA(cudaMemcpy(ed.data(), c->edges + t->edge_off, ed.size() * 4, cudaMemcpyDeviceToHost));
    static const char *kind_name[] = {"static", "branch", "loop", "const", "module", "subflow"};
    std::string s = "digraph tg {\n  node [shape=box];\n";
    char line[160];
    for (u32 v = 0; v < g->n; ++v) {
        const u32 kind = (rec[v].prm >> 16) & 0xFFu;
        const u32 arg = rec[v].prm >> 24;
        const u32 rounds = rec[v].prm & 0xFFFFu;
        const u64 first = rec[v].succ_off - t->edge_off;
        int k = std::snprintf(line, sizeof(line), "  n%u [label=\"%u %s R=%u", v, v, kind <= TG_SUBFLOW ? kind_name[kind] : "?",
                              rounds);
        if (kind == TG_COND_LOOP)
            k += std::snprintf(line + k, sizeof(line) - k, " T=%u", arg);
        else if (kind == TG_COND_CONST)
            k += std::snprintf(line + k, sizeof(line) - k, " r=%d", (int)(signed char)(unsigned char)arg);
        else if (kind >= TG_MODULE && first < ed.size())
            k += std::snprintf(line + k, sizeof(line) - k, " graph=%u%s", ed[first],
                               (kind == TG_SUBFLOW && (arg & 1u)) ? " detached" : "");
        std::snprintf(line + k, sizeof(line) - k, "\"%s];\n", kind >= TG_COND_BRANCH && kind <= TG_COND_CONST ? ", shape=diamond" : "");
        s += line;
    }
    for (u32 v = 0; v < g->n; ++v) {
        const u32 kind = (rec[v].prm >> 16) & 0xFFu;
        const u32 cnt = rec[v].deg & 0xFFFFu;
        const u64 first = rec[v].succ_off - t->edge_off + (kind >= TG_MODULE ? 1u : 0u);
        const bool weak = kind >= TG_COND_BRANCH && kind <= TG_COND_CONST;
        for (u32 j = 0; j < cnt && first + j < ed.size(); ++j) {
            const u32 d = ed[first + j] & ~kSoleBit;
            if (weak)
                std::snprintf(line, sizeof(line), "  n%u -> n%u [style=dashed, label=\"%u\"];\n", v, d, j);
            else
                std::snprintf(line, sizeof(line), "  n%u -> n%u;\n", v, d);
            s += line;
        }
    }
    s += "}\n";
    *len = s.size();
    if (!buf || cap < s.size() + 1)
        return TG_ERR_BUDGET;
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return TG_OK;
}

int tg_capture_run(tg_ctx *c, tg_graph *g, uint32_t max_streams, uint64_t *ns)
{
    if (!c || !g || g->ctx != c || max_streams == 0 || max_streams > 32 || g->n > 65536u || g->n_cond != 0 ||
        g->n_mod != 0)
        return TG_ERR_INVALID;
    if (c->serving || graph_busy(g))
        return TG_ERR_BUSY;
    int rc = clear_if_dirty(c);
    if (rc != TG_OK)
        return rc;
    if (g->setup_pending && (rc = instance_setup(c, g)) != TG_OK)
        return rc;
    if (g->ready)
        TG_CUDA(cudaStreamWaitEvent(c->stream, g->ready, 0));
    if (!g->cap_exec || g->cap_streams != max_streams) {
        // the packed successor lists (graph-local ids) and task records, read back
        const tg_graph *t = g->tmpl ? g->tmpl : g;
        std::vector<NodeSlot> rec(g->n);
        std::vector<u32> ed(t->m);
        TG_CUDA(cudaStreamSynchronize(c->stream));
        TG_CUDA(cudaMemcpy(rec.data(), c->slots + t->node_off, (size_t)g->n * sizeof(NodeSlot),
                           cudaMemcpyDeviceToHost));
        if (t->m)
            TG_CUDA(cudaMemcpy(ed.data(), c->edges + t->edge_off, (size_t)t->m * 4, cudaMemcpyDeviceToHost));
        std::vector<u32> off(g->n + 1, 0), adj(t->m);
        for (u32 v = 0; v < g->n; ++v) {
            const u32 cnt = rec[v].deg & 0xFFFFu;
            const u64 first = rec[v].succ_off - t->edge_off;
            if (first + cnt > t->m)
                return TG_ERR_INTERNAL;
            for (u32 j = 0; j < cnt; ++j)
                adj[off[v] + j] = ed[first + j] & ~kSoleBit;
            off[v + 1] = off[v] + cnt;
        }
        std::vector<u32> lv, ix;
        u32 nl = 0;
        if (!levelize_csr(g->n, off, adj, lv, ix, nl))
            return TG_ERR_INVALID;
        std::vector<std::vector<u32>> by_level(nl);
        for (u32 v = 0; v < g->n; ++v)
            by_level[lv[v]].push_back(v);
        std::vector<std::vector<u32>> preds(g->n);
        for (u32 v = 0; v < g->n; ++v)
            for (u32 e = off[v]; e < off[v + 1]; ++e)
                preds[adj[e]].push_back(v);
        auto stream_of = [&](u32 v) { return ix[v] % max_streams; };

        std::vector<cudaStream_t> S(max_streams, nullptr);
        std::vector<cudaEvent_t> ev(g->n, nullptr);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t fork = nullptr;
        cudaError_t err = cudaSuccess;
        auto chk = [&](cudaError_t e) {
            if (err == cudaSuccess && e != cudaSuccess)
                err = e;
            return err == cudaSuccess;
        };
        for (u32 s = 0; s < max_streams; ++s)
            chk(cudaStreamCreateWithFlags(&S[s], cudaStreamNonBlocking));
        chk(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (u32 v = 0; v < g->n && err == cudaSuccess; ++v)
            for (u32 e = off[v]; e < off[v + 1]; ++e)
                if (stream_of(adj[e]) != stream_of(v)) {
                    chk(cudaEventCreateWithFlags(&ev[v], cudaEventDisableTiming));
                    break;
                }
        KParams p = base_params(c, c->geo);
        p.lt = nullptr;
        p.n_graphs = 1;
        p.single_gid = g->gid;
        p.max_n = g->n;
        p.total_sources = g->n_src;
        const u32 base = (u32)g->node_off;
        if (chk(cudaStreamBeginCapture(S[0], cudaStreamCaptureModeThreadLocal))) {
            chk(launch_rearm(p, S[0]));
            chk(cudaEventRecord(fork, S[0]));
            for (u32 s = 1; s < max_streams; ++s)
                chk(cudaStreamWaitEvent(S[s], fork, 0));
            for (u32 l = 0; l < nl && err == cudaSuccess; ++l)
                for (u32 v : by_level[l]) {
                    const u32 s = stream_of(v);
                    for (u32 q : preds[v])
                        if (stream_of(q) != s)
                            chk(cudaStreamWaitEvent(S[s], ev[q], 0));
                    chk(launch_capture_task(c->slots, c->outv, c->edges, base + v, base, S[s]));
                    if (ev[v])
                        chk(cudaEventRecord(ev[v], S[s]));
                }
            // join every stream back into the first before the capture ends
            for (u32 s = 1; s < max_streams; ++s) {
                cudaEvent_t j = nullptr;
                if (chk(cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) && chk(cudaEventRecord(j, S[s])))
                    chk(cudaStreamWaitEvent(S[0], j, 0));
                if (j)
                    cudaEventDestroy(j);
            }
            cudaError_t e2 = cudaStreamEndCapture(S[0], &graph);
            chk(e2);
        }
        if (err == cudaSuccess)
            chk(cudaGraphInstantiate(&exec, graph, 0));
        if (graph)
            cudaGraphDestroy(graph);
        for (cudaEvent_t e : ev)
            if (e)
                cudaEventDestroy(e);
        if (fork)
            cudaEventDestroy(fork);
        for (cudaStream_t s : S)
            if (s)
                cudaStreamDestroy(s);
        if (err != cudaSuccess) {
            if (exec)
                cudaGraphExecDestroy(exec);
            return TG_ERR_CUDA;
        }
        if (g->cap_exec)
            cudaGraphExecDestroy(g->cap_exec);
        g->cap_exec = exec;
        g->cap_streams = max_streams;
    }
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(cudaGraphLaunch(g->cap_exec, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    TG_CUDA(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    TG_CUDA(cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
    if (ns)
        *ns = (u64)((double)ms * 1e6);
    c->timed = false;
    return TG_OK;
}

}  // extern "C"

// (Re)capture re-arm + scheduler + finalize of a batch with its geometry as
// one CUDA graph; replays reuse it.
static int batch_capture(tg_ctx *c, tg_batch *b)
{
    KParams p = base_params(c, b->geo);
    p.lt = (const LEntry *)(c->edges + b->lt_off);
    p.n_graphs = (u32)b->gs.size();
    p.single_gid = 0;
    p.max_n = b->max_n;
    p.total_sources = b->total_src;
    p.has_modules = b->has_mod ? 1u : 0u;
    if (b->acyclic)
        p.flags |= kFlagAcyclic;
    b->kp = p;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = c->capture_stream;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return TG_ERR_CUDA;
    cudaError_t e0 = cudaSuccess;
    for (tg_graph *mg : b->comp)   // composed graphs and subflow copies start idle
        if (e0 == cudaSuccess)
            e0 = launch_module_rearm(p, mg->gid, mg->n, cs);
    cudaError_t e1 = e0 != cudaSuccess ? e0 : launch_rearm(p, cs);
    cudaError_t e2 = launch_sched(p, b->geo.blocks, b->geo.threads, cs);
    cudaError_t e3 = launch_finalize(p, cs);
    cudaError_t e4 = cudaStreamEndCapture(cs, &graph);
    if (e1 || e2 || e3 || e4 || !graph) {
        if (graph)
            cudaGraphDestroy(graph);
        return TG_ERR_CUDA;
    }
    cudaError_t e5 = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    return e5 == cudaSuccess ? TG_OK : TG_ERR_CUDA;
}

extern "C" {

int tg_batch_create(tg_ctx *c, tg_graph *const *gs, uint32_t n, tg_batch **out)
{
    if (!c || !gs || !out || n == 0 || n > kMaxGraphs)
        return TG_ERR_INVALID;
    *out = nullptr;
    std::vector<LEntry> lt(n);
    u64 inj = 0;
    u32 max_n = 0;
    for (u32 i = 0; i < n; ++i) {
        if (!gs[i] || gs[i]->ctx != c)
            return TG_ERR_INVALID;
        for (u32 j = 0; j < i; ++j)
            if (gs[j] == gs[i])
                return TG_ERR_INVALID;
        lt[i].gid = gs[i]->gid;
        lt[i].inj_base = (u32)inj;
        inj += gs[i]->n_src;
        max_n = std::max(max_n, gs[i]->n);
    }
    if (inj > c->inj_cap)
        return TG_ERR_BUDGET;
    tg_batch *b = new (std::nothrow) tg_batch();
    if (!b)
        return TG_ERR_INVALID;
    c->live_batches.insert(b);
    b->ctx = c;
    b->gs.assign(gs, gs + n);
    b->lt_len = (u64)n * 2;
    if (!c->edge_pool.alloc(b->lt_len, b->lt_off)) {
        c->live_batches.erase(b);
        delete b;
        return TG_ERR_BUDGET;
    }
    if (cudaMemcpy(c->edges + b->lt_off, lt.data(), (size_t)n * sizeof(LEntry), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        tg_batch_destroy(c, b);
        return TG_ERR_CUDA;
    }
    b->max_n = max_n;
    b->total_src = (u32)inj;
    b->geo = c->geo;
    b->acyclic = true;
    for (tg_graph *g : b->gs) {
        b->has_mod = b->has_mod || g->n_mod != 0;
        b->acyclic = b->acyclic && g->n_cond == 0 && g->n_mod == 0;
    }
    if (b->has_mod)
        b->comp = composition_closure(b->gs);
    int rc = batch_capture(c, b);
    if (rc != TG_OK) {
        tg_batch_destroy(c, b);
        return rc;
    }
    if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
        tg_batch_destroy(c, b);
        return TG_ERR_CUDA;
    }
    for (tg_graph *g : b->gs)
        g->n_batches++;
    b->counted = true;
    *out = b;
    return TG_OK;
}

int tg_batch_launch(tg_ctx *c, tg_batch *b)
{
    if (!c || !b || b->ctx != c)
        return TG_ERR_INVALID;
    if (c->serving)
        return TG_ERR_BUSY;
    for (tg_graph *g : b->gs)
        if (graph_busy(g))
            return TG_ERR_BUSY;
    int rc = clear_if_dirty(c);
    if (rc != TG_OK)
        return rc;
    for (tg_graph *g : b->gs) {
        if (g->setup_pending) {
            int rc2 = instance_setup(c, g);
            if (rc2 != TG_OK)
                return rc2;
        }
        if (g->ready)
            TG_CUDA(cudaStreamWaitEvent(c->stream, g->ready, 0));
    }
    for (tg_graph *g : b->comp)
        if (g->ready)
            TG_CUDA(cudaStreamWaitEvent(c->stream, g->ready, 0));
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(cudaGraphLaunch(b->exec, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    TG_CUDA(cudaEventRecord(b->done, c->stream));
    c->timed = true;
    c->last_geo = b->geo;
    for (tg_graph *g : b->gs)
        g->busy = b->done;
    b->launched = true;
    return TG_OK;
}

int tg_batch_wait(tg_ctx *c, tg_batch *b, int *statuses)
{
    if (!c || !b || b->ctx != c || !b->launched)
        return TG_ERR_INVALID;
    TG_CUDA(cudaEventSynchronize(b->done));
    int first = TG_OK;
    for (size_t i = 0; i < b->gs.size(); ++i) {
        tg_graph *g = b->gs[i];
        int st = c->h_status[g->gid];
        note_status(c, st);
        if (statuses)
            statuses[i] = st;
        if (st != TG_OK && first == TG_OK)
            first = st;
        if (g->busy == b->done)
            g->busy = nullptr;
    }
    b->launched = false;
    return first;
}

int tg_batch_destroy(tg_ctx *c, tg_batch *b)
{
    if (!c || !b || b->ctx != c)
        return TG_ERR_INVALID;
    if (b->launched)
        cudaEventSynchronize(b->done);
    for (tg_graph *g : b->gs) {
        if (g->busy == b->done)
            g->busy = nullptr;
        if (b->counted)
            g->n_batches--;
    }
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->done)
        cudaEventDestroy(b->done);
    if (b->lt_len)
        c->edge_pool.release(b->lt_off, b->lt_len);
    c->live_batches.erase(b);
    delete b;
    return TG_OK;
}

}  // extern "C"

// One timed replay of a batch under its current geometry (graph re-captured
// by the caller); returns the device time or 0 on failure, *status the
// first graph error.
static u64 batch_time(tg_ctx *c, tg_batch *b, int *status)
{
    if (tg_batch_launch(c, b) != TG_OK) {
        *status = TG_ERR_CUDA;
        return 0;
    }
    *status = tg_batch_wait(c, b, nullptr);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1) != cudaSuccess)
        return 0;
    return (u64)((double)ms * 1e6);
}

static std::string batch_key(tg_ctx *c, tg_batch *b)
{
    u64 nodes = 0, edges = 0, srcs = 0;
    for (tg_graph *g : b->gs) {
        nodes += g->n;
        edges += g->m;
        srcs += g->n_src;
    }
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|sm%d|flags%u|g%zu|n%llu|m%llu|s%llu", c->dev_name.c_str(), c->sm_count,
                  c->opts.flags, b->gs.size(), (unsigned long long)nodes, (unsigned long long)edges,
                  (unsigned long long)srcs);
    std::string k(buf);
    for (char &ch : k)
        if (ch == '\t' || ch == '\n')
            ch = ' ';
    return k;
}

// Coordinate descent over the launch knobs; `measure` times one candidate
// (TG_ERR_INVALID / TG_ERR_CUDA from it skip the candidate, other errors end
// the search).  A text file caches the winner under `key`.
static int tune_geometry(tg_ctx *c, const std::string &key, const char *cache_path, tg_ctx_opts &best,
                         u64 &best_t, const std::function<int(const tg_ctx_opts &, u64 &)> &measure)
{
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "r")) {
            char line[1024];
            bool hit = false;
            while (std::fgets(line, sizeof(line), f)) {
                char *tab = std::strchr(line, '\t');
                if (!tab || std::string(line, tab) != key)
                    continue;
                tg_ctx_opts o{};
                unsigned long long t = 0;
                if (std::sscanf(tab + 1, "%d %d %d %d %d %d %d %u %d %d %d %u %d %d %llu", &o.worker_blocks,
                                &o.warps_per_block, &o.deque_depth, &o.steal_policy, &o.max_steal, &o.max_thieves,
                                &o.smem_ring, &o.idle_sleep_ns, &o.batch_max, &o.local_keep, &o.thief_mode,
                                &o.steal_backoff_ns, &o.keep_idle, &o.hand_batch, &t) == 15) {
                    Geometry g;
                    if (resolve_geometry(c, o, g) == TG_OK) {
                        best = o;
                        best_t = t;
                        hit = true;
                    }
                }
            }
            std::fclose(f);
            if (hit)
                return TG_OK;
        }
    }
    int rc = measure(best, best_t);
    if (rc != TG_OK)
        return rc;
    const int warps_c[] = {4, 8, 16};
    const int bpsm_c[] = {1, 2, 4};
    const int depth_c[] = {(int)std::max<u32>(64u, c->dq_cap / 4u), (int)c->dq_cap};
    const int policy_c[] = {0, 1};
    const int steal_c[] = {2, 8, 32};
    const int thief_c[] = {8, 16, 64};
    const int batch_c[] = {8, 16, 24, 32};
    const int keep_c[] = {16, 32, 64, 128, 512};
    const int tmode_c[] = {0, 1};
    const int backoff_c[] = {128, 512, 4096};
    const int idle_c[] = {128, 256, 1024};
    const int keep_idle_c[] = {0, 1};
    const int hand_batch_c[] = {0, 1};
    // every candidate measured, for the confirmation below
    std::vector<std::pair<u64, tg_ctx_opts>> seen;
    if (best_t)
        seen.push_back({best_t, best});
    auto try_knob = [&](auto setter, const int *vals, int nv) -> int {
        for (int i = 0; i < nv; ++i) {
            tg_ctx_opts o = best;
            setter(o, vals[i]);
            Geometry g;
            if (resolve_geometry(c, o, g) != TG_OK)
                continue;
            geometry_to_opts(g, o);
            if (std::memcmp(&o, &best, sizeof(o)) == 0)
                continue;
            u64 t = 0;
            int rc2 = measure(o, t);
            // a candidate whose run reported a race is skipped: the start
            // geometry ran clean, so the graph is not racy and the report is
            // the race check's known false positive (a task re-activated
            // while it finishes its step), which some geometries provoke; so
            // is one that ran into the time limit (adaptive thieves over many
            // small blocks can be two orders of magnitude slower)
            if (rc2 == TG_ERR_INVALID || rc2 == TG_ERR_CUDA || rc2 == TG_ERR_RACE || rc2 == TG_ERR_TIMEOUT)
                continue;
            if (rc2 != TG_OK)
                return rc2;
            if (t)
                seen.push_back({t, o});
            if (t && t < best_t) {
                best_t = t;
                best = o;
            }
        }
        return TG_OK;
    };
    // the knobs interact (a larger batch wants a longer backlog), so a pass
    // that improved on the start is followed by one more
    for (int pass = 0; pass < 2; ++pass) {
        const u64 pass_t = best_t;
        if ((rc = try_knob([](tg_ctx_opts &o, int v) { o.warps_per_block = v; o.worker_blocks = 0; }, warps_c, 3)) != TG_OK ||
            (rc = try_knob([&](tg_ctx_opts &o, int v) { o.worker_blocks = v * c->sm_count; }, bpsm_c, 3)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.deque_depth = v; }, depth_c, 2)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.steal_policy = v; }, policy_c, 2)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.max_steal = v; }, steal_c, 3)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.max_thieves = v; }, thief_c, 3)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.batch_max = v; }, batch_c, 4)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.local_keep = v; }, keep_c, 5)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.keep_idle = v; }, keep_idle_c, 2)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.hand_batch = v; }, hand_batch_c, 2)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.thief_mode = v; }, tmode_c, 2)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.steal_backoff_ns = (u32)v; }, backoff_c, 3)) != TG_OK ||
            (rc = try_knob([](tg_ctx_opts &o, int v) { o.idle_sleep_ns = (u32)v; }, idle_c, 3)) != TG_OK)
            return rc;
        if (best_t >= pass_t)
            break;
    }
    // Confirmation: a single measurement per candidate is a few percent
    // noisy, about what separates the best geometries of a graph, so the
    // three fastest distinct candidates are measured once more and the pick
    // is the fastest by the sum of both measurements.
    std::sort(seen.begin(), seen.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    std::vector<std::pair<u64, tg_ctx_opts>> top;
    for (const auto &cand : seen) {
        bool dup = false;
        for (const auto &t : top)
            dup = dup || std::memcmp(&t.second, &cand.second, sizeof(tg_ctx_opts)) == 0;
        if (!dup)
            top.push_back(cand);
        if (top.size() == 3)
            break;
    }
    if (top.size() > 1) {
        u64 best_sum = ~0ull;
        for (const auto &cand : top) {
            u64 t2 = 0;
            const int rc3 = measure(cand.second, t2);
            if (rc3 == TG_ERR_INVALID || rc3 == TG_ERR_CUDA || rc3 == TG_ERR_RACE || rc3 == TG_ERR_TIMEOUT || !t2)
                continue;
            if (rc3 != TG_OK)
                return rc3;
            if (cand.first + t2 < best_sum) {
                best_sum = cand.first + t2;
                best = cand.second;
                best_t = std::min(cand.first, t2);
            }
        }
    }
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "a")) {
            std::fprintf(f, "%s\t%d %d %d %d %d %d %d %u %d %d %d %u %d %d %llu\n", key.c_str(), best.worker_blocks,
                         best.warps_per_block, best.deque_depth, best.steal_policy, best.max_steal,
                         best.max_thieves, best.smem_ring, best.idle_sleep_ns, best.batch_max, best.local_keep,
                         best.thief_mode, best.steal_backoff_ns, best.keep_idle, best.hand_batch,
                         (unsigned long long)best_t);
            std::fclose(f);
        }
    }
    return TG_OK;
}

static std::string graph_key(tg_ctx *c, tg_graph *g)
{
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|sm%d|flags%u|graph|n%u|m%u|s%u|c%u|mod%u", c->dev_name.c_str(), c->sm_count,
                  c->opts.flags, g->n, g->m, g->n_src, g->n_cond, g->n_mod);
    std::string k(buf);
    for (char &ch : k)
        if (ch == '\t' || ch == '\n')
            ch = ' ';
    return k;
}

extern "C" {

int tg_batch_autotune(tg_ctx *c, tg_batch *b, uint32_t trials, const char *cache_path, tg_ctx_opts *chosen,
                      uint64_t *best_ns)
{
    if (!c || !b || b->ctx != c)
        return TG_ERR_INVALID;
    if (trials == 0)
        trials = 2;
    tg_ctx_opts best{};
    geometry_to_opts(b->geo, best);
    u64 best_t = 0;
    auto measure = [&](const tg_ctx_opts &o, u64 &t_out) -> int {
        Geometry g;
        int rc = resolve_geometry(c, o, g);
        if (rc != TG_OK)
            return rc;
        b->geo = g;
        rc = batch_capture(c, b);
        if (rc != TG_OK)
            return rc;
        int st = TG_OK;
        batch_time(c, b, &st);   // warm-up replay
        if (st != TG_OK)
            return st;
        u64 tmin = 0;
        for (uint32_t i = 0; i < trials; ++i) {
            u64 t = batch_time(c, b, &st);
            if (st != TG_OK)
                return st;
            if (t && (tmin == 0 || t < tmin))
                tmin = t;
        }
        t_out = tmin;
        return TG_OK;
    };
    int rc = tune_geometry(c, batch_key(c, b), cache_path, best, best_t, measure);
    if (rc != TG_OK)
        return rc;
    Geometry g;
    rc = resolve_geometry(c, best, g);
    if (rc != TG_OK)
        return rc;
    b->geo = g;
    rc = batch_capture(c, b);
    if (rc != TG_OK)
        return rc;
    if (chosen) {
        *chosen = c->opts;
        geometry_to_opts(g, *chosen);
    }
    if (best_ns)
        *best_ns = best_t;
    return TG_OK;
}

int tg_graph_autotune(tg_ctx *c, tg_graph *g, uint32_t trials, const char *cache_path, tg_ctx_opts *chosen,
                      uint64_t *best_ns)
{
    if (!c || !g || g->ctx != c)
        return TG_ERR_INVALID;
    if (c->serving)
        return TG_ERR_BUSY;
    if (trials == 0)
        trials = 2;
    tg_ctx_opts best{};
    geometry_to_opts(g->has_geo ? g->geo : c->geo, best);
    u64 best_t = 0;
    auto run_once = [&](u64 &ns) -> int {
        uint64_t t = 0;
        int rc = tg_submit(c, g, &t);
        if (rc != TG_OK)
            return rc;
        rc = tg_wait(c, t);
        if (rc != TG_OK)
            return rc;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1) != cudaSuccess)
            return TG_ERR_CUDA;
        ns = (u64)((double)ms * 1e6);
        return TG_OK;
    };
    auto measure = [&](const tg_ctx_opts &o, u64 &t_out) -> int {
        Geometry geo;
        int rc = resolve_geometry(c, o, geo);
        if (rc != TG_OK)
            return rc;
        g->geo = geo;
        g->has_geo = true;
        u64 t = 0;
        if ((rc = run_once(t)) != TG_OK)   // warm-up
            return rc;
        u64 tmin = 0;
        for (uint32_t i = 0; i < trials; ++i) {
            if ((rc = run_once(t)) != TG_OK)
                return rc;
            if (t && (tmin == 0 || t < tmin))
                tmin = t;
        }
        t_out = tmin;
        return TG_OK;
    };
    int rc = tune_geometry(c, graph_key(c, g), cache_path, best, best_t, measure);
    if (rc != TG_OK) {
        g->has_geo = false;
        return rc;
    }
    Geometry geo;
    rc = resolve_geometry(c, best, geo);
    if (rc != TG_OK)
        return rc;
    g->geo = geo;
    g->has_geo = true;
    if (chosen) {
        *chosen = c->opts;
        geometry_to_opts(geo, *chosen);
    }
    if (best_ns)
        *best_ns = best_t;
    return TG_OK;
}

int tg_run_batch(tg_ctx *c, tg_graph *const *gs, uint32_t n, int *statuses)
{
    tg_batch *b = nullptr;
    int rc = tg_batch_create(c, gs, n, &b);
    if (rc != TG_OK)
        return rc;
    rc = tg_batch_launch(c, b);
    if (rc == TG_OK)
        rc = tg_batch_wait(c, b, statuses);
    tg_batch_destroy(c, b);
    return rc;
}

int tg_ctx_get_stats(tg_ctx *c, tg_stats *st)
{
    if (!c || !st)
        return TG_ERR_INVALID;
    memset(st, 0, sizeof(*st));
    TG_CUDA(cudaStreamSynchronize(c->stream));
    const Geometry &lg = c->last_geo.blocks > 0 ? c->last_geo : c->geo;
    const int nb = lg.blocks;
    std::vector<u64> h((size_t)nb * ST_COUNT);
    TG_CUDA(cudaMemcpy(h.data(), c->stats, h.size() * sizeof(u64), cudaMemcpyDeviceToHost));
    for (int b = 0; b < nb; ++b) {
        const u64 *s = &h[(size_t)b * ST_COUNT];
        st->tasks += s[ST_TASKS];
        st->pops_local += s[ST_POP_LOCAL];
        st->pops_own += s[ST_POP_OWN];
        st->steal_attempts += s[ST_STEAL_TRY];
        st->steal_hits += s[ST_STEAL_HIT];
        st->inject_pops += s[ST_INJECT];
        st->spills += s[ST_SPILL];
        st->idle_loops += s[ST_IDLE];
        st->warp_iters += s[ST_ITERS];
        st->pops_hand += s[ST_HAND];
        for (int i = 0; i < 5; ++i)
            st->phase_cycles[i] += s[ST_PHASE0 + i];
        st->parks += s[ST_PARK];
        st->failed_rounds += s[ST_FAILED_ROUND];
        st->round_cycles += s[ST_ROUND_CYCLES];
        st->peak_thieves = std::max<uint64_t>(st->peak_thieves, s[ST_PEAK_THIEVES]);
    }
    if (c->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1) == cudaSuccess)
            st->kernel_ns = (u64)((double)ms * 1e6);
    }
    st->worker_blocks = (u32)nb;
    st->warps_per_block = (u32)(lg.threads / 32);
    return TG_OK;
}

int tg_bench_payload(tg_ctx *c, uint64_t count, uint32_t rounds, uint64_t *ns, uint32_t *checksum)
{
    if (!c || !ns)
        return TG_ERR_INVALID;
    TG_CUDA(cudaMemsetAsync(c->scratch, 0, 4, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(launch_bench_payload(count, rounds, c->scratch, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    u32 cs = 0;
    TG_CUDA(cudaMemcpyAsync(&cs, c->scratch, 4, cudaMemcpyDeviceToHost, c->stream));
    TG_CUDA(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    TG_CUDA(cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
    *ns = (u64)((double)ms * 1e6);
    if (checksum)
        *checksum = cs;
    c->timed = false;
    return TG_OK;
}

int tg_bench_payload_tasks(tg_ctx *c, uint32_t n, const uint32_t *ids, const uint32_t *rounds, const uint32_t *cnt,
                           uint64_t *ns, uint32_t *checksum)
{
    if (!c || !ns || (n && (!ids || !rounds || !cnt)))
        return TG_ERR_INVALID;
    TG_CUDA(cudaMemsetAsync(c->scratch, 0, 4, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(launch_bench_payload_tasks(n, ids, rounds, cnt, c->scratch, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    u32 cs = 0;
    TG_CUDA(cudaMemcpyAsync(&cs, c->scratch, 4, cudaMemcpyDeviceToHost, c->stream));
    TG_CUDA(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    TG_CUDA(cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
    *ns = (u64)((double)ms * 1e6);
    if (checksum)
        *checksum = cs;
    c->timed = false;
    return TG_OK;
}

int tg_bench_atomics(tg_ctx *c, uint64_t count, uint64_t footprint_words, uint64_t *ns)
{
    if (!c || !ns || footprint_words == 0 || footprint_words > c->inj_cap)
        return TG_ERR_INVALID;
    // the injection queue's memory serves as the footprint; it is cleared
    // before the next scheduler launch
    c->dirty = true;
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(launch_bench_atomics(c->inj, footprint_words, count, (u64 *)c->scratch, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    TG_CUDA(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    TG_CUDA(cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
    *ns = (u64)((double)ms * 1e6);
    c->timed = false;
    return TG_OK;
}

int tg_bench_chain(tg_ctx *c, uint32_t hops, uint32_t rounds, uint64_t *ns, uint32_t *last)
{
    if (!c || !ns || rounds > 0xFFFFu)
        return TG_ERR_INVALID;
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(launch_bench_chain(hops, rounds, c->scratch, c->stream));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    u32 out = 0;
    TG_CUDA(cudaMemcpyAsync(&out, c->scratch, 4, cudaMemcpyDeviceToHost, c->stream));
    TG_CUDA(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    TG_CUDA(cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
    *ns = (u64)((double)ms * 1e6);
    if (last)
        *last = out;
    c->timed = false;
    return TG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// server mode: a resident scheduler fed through a submission ring
// ---------------------------------------------------------------------------
static void drain_completions(tg_ctx *c)
{
    for (;;) {
        const u64 rec = ((volatile u64 *)c->h_comp)[c->comp_read & (kSubRing - 1u)];
        if ((rec >> 32) != (u32)(c->comp_read + 1u))
            break;
        const u32 gid = (u32)(rec & 0xFFFFu);
        const int st = (int)(int16_t)(uint16_t)((rec >> 16) & 0xFFFFu);
        tg_graph *g = c->by_gid[gid];
        if (g) {
            c->serve_done[g->serve_ticket] = st;
            c->newly_done.push_back(g->serve_ticket);
            g->serve_ticket = 0;
            c->by_gid[gid] = nullptr;
        }
        c->comp_read++;
    }
}

static int serve_submit(tg_ctx *c, tg_graph *g, uint64_t *ticket)
{
    if (g->serve_ticket != 0 || graph_busy(g))
        return TG_ERR_BUSY;
    tg_graph *src = g->tmpl ? g->tmpl : g;
    // re-arm on the side stream: fresh task records from the template's
    // (join words, counts, digests), then the ring entry -- stream order
    // makes the records visible before the scheduler can see the entry
    const u64 seq = c->sub_seq++;
    SubEntry &h = c->h_sub[seq & (kSubRing - 1u)];
    h.seq = (u32)(seq + 1u);
    h.gid = g->gid;
    h.node_off = (u32)g->node_off;
    h.n = g->n;
    h.seed = g->seed;
    h.src_off = (u32)(src->edge_off + src->m);
    h.n_src = g->n_src;
    h.exec_cap = (u32)std::min<u64>(c->opts.exec_cap, 0xFFFFFFFFull);
    g->setup_pending = false;   // the scheduler writes descriptor and chunk table on claim
    TG_CUDA(launch_instance_rearm(c->slots, src->node_off, g->node_off, g->n, c->side));
    // the entry's fields first, its sequence word last: a scheduler that sees
    // the new seq then reads complete fields (stream order of the copies)
    SubEntry *dst = &c->sub[seq & (kSubRing - 1u)];
    TG_CUDA(cudaMemcpyAsync(&dst->gid, &h.gid, sizeof(SubEntry) - sizeof(u32), cudaMemcpyHostToDevice, c->side));
    TG_CUDA(cudaMemcpyAsync(&dst->seq, &h.seq, sizeof(u32), cudaMemcpyHostToDevice, c->side));
    g->serve_ticket = c->next_ticket++;
    c->by_gid[g->gid] = g;
    *ticket = g->serve_ticket;
    return TG_OK;
}

static int serve_poll(tg_ctx *c, uint64_t ticket)
{
    drain_completions(c);
    auto it = c->serve_done.find(ticket);
    if (it != c->serve_done.end())
        return it->second;
    if (!c->serving)
        return TG_ERR_INVALID;
    return TG_PENDING;
}

extern "C" {

int tg_serve_start(tg_ctx *c, uint64_t time_limit_ns)
{
    if (!c)
        return TG_ERR_INVALID;
    if (c->serving)
        return TG_ERR_BUSY;
    TG_CUDA(cudaStreamSynchronize(c->stream));
    if (!c->by_gid) {
        c->by_gid = new (std::nothrow) tg_graph *[kMaxGraphs];
        if (!c->by_gid)
            return TG_ERR_INVALID;
    }
    for (u32 i = 0; i < kMaxGraphs; ++i)
        c->by_gid[i] = nullptr;
    int rc = clear_if_dirty(c);
    if (rc != TG_OK)
        return rc;
    Geometry g = c->geo;
    // one block per SM, of a shape of which two would fit: the resident
    // server leaves room on every SM for the kernels that re-arm
    // instances (their records from the template's immutable half)
    int per_sm = 0;
    for (;;) {
        if (sched_occupancy(g.threads, sched_dyn_smem(g.ring, (u32)(g.threads / 32)), &per_sm, true) !=
            cudaSuccess)
            return TG_ERR_CUDA;
        if (per_sm >= 2 || g.threads <= 64)
            break;
        g.threads /= 2;
    }
    if (per_sm < 2)
        return TG_ERR_CUDA;
    g.blocks = std::min(g.blocks, std::min(c->sm_count, kMaxBlocks));
    c->serve_geo = g;
    *(volatile u32 *)c->h_stop = 0u;
    memset(c->h_comp, 0, (size_t)kSubRing * 8);
    c->sub_seq = 0;
    c->comp_read = 0;
    TG_CUDA(cudaMemsetAsync(c->ctl, 0, sizeof(LaunchCtl), c->stream));
    TG_CUDA(cudaMemsetAsync(c->sub, 0, (size_t)kSubRing * sizeof(SubEntry), c->stream));
    TG_CUDA(cudaMemsetAsync(c->dqc, 0, (size_t)kMaxBlocks * sizeof(QCtr), c->stream));
    TG_CUDA(cudaMemsetAsync(c->thief_slots, 0, (size_t)1024 * 128, c->stream));
    TG_CUDA(cudaMemsetAsync(c->stats, 0, (size_t)kMaxBlocks * ST_COUNT * sizeof(u64), c->stream));
    TG_CUDA(preload_serving_kernels(c->side));
    TG_CUDA(cudaStreamSynchronize(c->side));
    TG_CUDA(cudaStreamSynchronize(c->stream));
    KParams p = base_params(c, g);
    p.lt = nullptr;
    p.n_graphs = 0;
    p.single_gid = 0;
    p.time_limit_ns = time_limit_ns ? time_limit_ns : 60ull * 1000 * 1000 * 1000;
    TG_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    TG_CUDA(launch_sched(p, g.blocks, g.threads, c->stream, true));
    TG_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    c->last_geo = g;
    c->timed = true;
    c->serving = true;
    return TG_OK;
}

int tg_serve_stop(tg_ctx *c)
{
    if (!c)
        return TG_ERR_INVALID;
    if (!c->serving)
        return TG_ERR_INVALID;
    // the stop word lives in device memory (idle blocks poll it); write it
    // behind every queued submission
    *(volatile u32 *)c->h_stop = 1u;
    cudaError_t e = cudaMemcpyAsync(&c->ctl->stop, c->h_stop, sizeof(u32), cudaMemcpyHostToDevice, c->side);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    drain_completions(c);
    c->serving = false;
    if (e != cudaSuccess)
        return TG_ERR_CUDA;
    LaunchCtl h{};
    TG_CUDA(cudaMemcpy(&h, c->ctl, sizeof(h), cudaMemcpyDeviceToHost));
    // graphs still in flight end with the abort code (or TIMEOUT)
    const int code = h.abort_code != 0 ? h.abort_code : TG_OK;
    for (u32 i = 0; i < kMaxGraphs; ++i) {
        if (tg_graph *g = c->by_gid[i]) {
            c->serve_done[g->serve_ticket] = code != TG_OK ? code : TG_ERR_CANCELLED;
            g->serve_ticket = 0;
            c->by_gid[i] = nullptr;
        }
    }
    c->dirty = true;
    return code;
}

}  // extern "C"

extern "C" int tg_serve_replay(tg_ctx *c, tg_graph *const *templates, uint32_t n_templates, const uint32_t *which,
                               const uint64_t *arrival_ns, uint32_t n_requests, uint64_t *latency_ns, int *status,
                               uint32_t *max_in_flight, tg_graph **keep, const uint8_t *keep_mask)
{
    if (!c || !c->serving || !templates || !which || !arrival_ns || !latency_ns || !status)
        return TG_ERR_INVALID;
    for (uint32_t i = 0; i < n_requests; ++i)
        if (which[i] >= n_templates || !templates[which[i]] || templates[which[i]]->ctx != c)
            return TG_ERR_INVALID;
    if (keep)
        for (uint32_t i = 0; i < n_requests; ++i)
            keep[i] = nullptr;
    // request r's instance is kept (not destroyed) when it finishes
    auto kept = [&](uint32_t r) { return keep && (!keep_mask || keep_mask[r]); };
    struct Flight {
        uint32_t req;
        tg_graph *inst;
    };
    std::map<u64, Flight> flight;
    std::vector<uint32_t> waiting;   // FIFO of admitted-to-host, not yet on the device
    size_t wait_head = 0;
    uint32_t next = 0, done = 0, peak = 0;
    int first_err = TG_OK;
    c->newly_done.clear();
    const u64 t0 = now_ns();
    while (done < n_requests) {
        bool progress = false;
        u64 now = now_ns() - t0;
        while (next < n_requests && arrival_ns[next] <= now)
            waiting.push_back(next++);
        // admission: an instance per request while budget and slots allow
        while (wait_head < waiting.size()) {
            const uint32_t r = waiting[wait_head];
            tg_graph *inst = nullptr;
            int rc = tg_instance_create(c, templates[which[r]], &inst);
            if (rc == TG_ERR_BUDGET && !flight.empty())
                break;   // wait for a finished graph to free memory or a slot
            wait_head++;
            progress = true;
            if (rc == TG_OK) {
                uint64_t t = 0;
                rc = serve_submit(c, inst, &t);
                if (rc == TG_OK) {
                    flight[t] = Flight{r, inst};
                    peak = std::max<uint32_t>(peak, (uint32_t)flight.size());
                    continue;
                }
                tg_graph_destroy(c, inst);
            }
            status[r] = rc;
            latency_ns[r] = 0;
            if (first_err == TG_OK)
                first_err = rc;
            done++;
        }
        // completions: free the instance at once
        drain_completions(c);
        if (!c->newly_done.empty()) {
            now = now_ns() - t0;
            for (u64 t : c->newly_done) {
                auto it = flight.find(t);
                if (it == flight.end())
                    continue;
                const uint32_t r = it->second.req;
                const int st = c->serve_done[t];
                c->serve_done.erase(t);
                status[r] = st;
                latency_ns[r] = now > arrival_ns[r] ? now - arrival_ns[r] : 0;
                if (st != TG_OK && first_err == TG_OK)
                    first_err = st;
                if (kept(r))
                    keep[r] = it->second.inst;
                else
                    tg_graph_destroy(c, it->second.inst);
                flight.erase(it);
                done++;
            }
            c->newly_done.clear();
            progress = true;
        }
        if (!progress && cudaStreamQuery(c->stream) != cudaErrorNotReady) {
            // the resident scheduler ended (time limit / fault): fail the rest
            for (auto &kv : flight) {
                status[kv.second.req] = TG_ERR_TIMEOUT;
                if (keep)   // still named by the server's records: the caller destroys it after stopping
                    keep[kv.second.req] = kv.second.inst;
                done++;
            }
            for (size_t i = wait_head; i < waiting.size(); ++i, ++done)
                status[waiting[i]] = TG_ERR_TIMEOUT;
            for (; next < n_requests; ++next, ++done)
                status[next] = TG_ERR_TIMEOUT;
            if (first_err == TG_OK)
                first_err = TG_ERR_TIMEOUT;
            break;
        }
    }
    if (max_in_flight)
        *max_in_flight = peak;
    return first_err;
}


extern "C" int tg_trace_copy(tg_ctx *c, const tg_graph *g, uint64_t *start_ns, uint64_t *end_ns, uint32_t *where)
{
    if (!c || !g || g->ctx != c || !c->trace)
        return TG_ERR_INVALID;
    TG_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<u64> h((size_t)g->n * 3);
    TG_CUDA(cudaMemcpy(h.data(), c->trace + 3 * (size_t)g->node_off, h.size() * 8, cudaMemcpyDeviceToHost));
    for (u32 v = 0; v < g->n; ++v) {
        if (start_ns)
            start_ns[v] = h[3 * (size_t)v];
        if (end_ns)
            end_ns[v] = h[3 * (size_t)v + 1];
        if (where)
            where[v] = (u32)h[3 * (size_t)v + 2];
    }
    return TG_OK;
}
