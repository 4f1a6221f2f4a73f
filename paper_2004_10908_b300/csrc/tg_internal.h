// tg_internal.h -- device data layout shared by the host library (tg_host.cpp)
// and the kernels (tg_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tg {

using u8 = uint8_t;
using u32 = uint32_t;
using i32 = int32_t;
using u64 = unsigned long long;

// One task of a resident graph: 32 bytes = one L2 sector, so the immutable
// record and the mutable join/execution state arrive in a single read.
struct alignas(32) NodeSlot {
    u32 succ_off;   // first successor in the edge pool (global index)
    u32 deg;        // successor count (bits 0-15) | strong in-degree (bits 16-31)
    u32 prm;        // rounds (0-15) | kind (16-23) | arg (24-31): loop trip or constant index
    u32 lid;        // the task's id inside its graph (payload input)
    u64 W;          // join word: insum of the current round (hi 32) | remaining strong deps (lo 32)
    u32 cnt;        // executions so far (bits 0-30) | in-flight flag (bit 31)
    u32 dig;        // digest of all outputs
};
static_assert(sizeof(NodeSlot) == 32, "NodeSlot must be one sector");

// Per-graph descriptor (indexed by graph slot id "gid").
struct alignas(64) GDesc {
    u64 pe;         // executions (hi 32) | pending activations (lo 32)
    i32 status;     // 0 while running / ok, else TG_ERR_*
    u32 seed;       // condition-hash seed
    u32 node_off;   // first node slot
    u32 n;          // tasks
    u32 src_off;    // source list in the edge pool
    u32 n_src;
    u32 exec_cap;
    u32 ret;        // composed graph in use: the module task to resume when it completes (else kEmpty32)
    u32 acc;        // subflow copy: sum of its sink outputs in the current spawn
    u32 pad[5];
};
static_assert(sizeof(GDesc) == 64, "GDesc is 64 bytes");

// One graph of a launch: its slot id and where its sources start in the
// injection queue.
struct LEntry {
    u32 gid;
    u32 inj_base;
};

// Head / tail of a multi-producer multi-consumer ring, on separate lines.
struct alignas(128) QCtr {
    u32 head;
    u32 pad0[31];
    u32 tail;
    u32 pad1[31];
};

// One submission of the server-mode ring: written by the host (copy engine),
// claimed by a thief when seq == its ticket + 1.
struct alignas(32) SubEntry {
    u32 seq;
    u32 gid;
    u32 node_off;
    u32 n;
    u32 seed;
    u32 src_off;
    u32 n_src;
    u32 exec_cap;
};

// Launch-wide control words (each on its own 128-byte line).
struct alignas(128) LaunchCtl {
    u32 graphs_left;
    u32 pad0[31];
    i32 abort_code;
    u32 pad1[31];
    u32 hungry;
    u32 pad2[31];
    QCtr inj;
    u32 avail[32];   // bit b: block b's public deque may hold work (blocks < 1024)
    u32 pad3[96];
    u32 sub_head;    // server mode: next submission to claim
    u32 pad4[31];
    u32 comp_tail;   // server mode: completion records written
    u32 pad5[31];
    u32 stop;        // server mode: set by the host (copy engine) to end the server
    u32 pad6[31];
    u32 actives;     // thief_mode 1: blocks with a warp executing work
    u32 pad7[31];
    u32 thieves;     // thief_mode 1: blocks stealing
    u32 pad8[31];
    u32 wake;        // thief_mode 1: wake tickets for parked blocks
    u32 pad9[31];
};

enum StatIdx {
    ST_TASKS = 0, ST_POP_LOCAL, ST_POP_OWN, ST_STEAL_TRY, ST_STEAL_HIT, ST_INJECT,
    ST_SPILL, ST_IDLE, ST_ITERS, ST_HAND, ST_PHASE0,   // ST_PHASE0 .. +4: traced cycles
    ST_PARK = ST_PHASE0 + 5, ST_PEAK_THIEVES, ST_FAILED_ROUND, ST_ROUND_CYCLES, ST_COUNT = 24
};

constexpr u32 kEmpty32 = 0xFFFFFFFFu;
constexpr u64 kEmpty = 0xFFFFFFFFFFFFFFFFull;
constexpr u32 kStrongBit = 0x80000000u;   // in a ready entry's low word
constexpr u32 kIdMask = 0x7FFFFFFFu;      // the task part of a ready entry's low word
constexpr u32 kInflight = 0x80000000u;    // in NodeSlot::cnt
constexpr u32 kAwait = 0x40000000u;       // in NodeSlot::cnt: a module task waits for its composed graph
constexpr u32 kDetachBit = 0x80000000u;   // in GDesc::ret: the copy of a detached subflow (holds a
                                          // token of its parent graph's pending count)
constexpr u32 kMaxNodeIndex = 0x7FFFFFFEu;
constexpr u32 kFlagAcyclic = 0x80000000u;  // in KParams::flags (set by the library, never by the
                                           // caller): no graph of the launch has condition,
                                           // module or subflow tasks, so every task runs once
constexpr u32 kSoleBit = 0x80000000u;     // in a static task's successor id: the target has
                                          // strong in-degree 1 (its join word is never used)
constexpr u32 kChunkShift = 8;            // node ranges are allocated in 256-task chunks
constexpr u32 kChunk = 1u << kChunkShift;

struct KParams {
    NodeSlot *slots;
    u32 *outv;
    const u32 *chunk_gid;  // graph slot of every 256-task chunk of the node pool
    const u32 *edges;      // successor lists and sources, as graph-local task ids
    GDesc *descs;
    const LEntry *lt;      // launch table (nullptr: single graph `single_gid`)
    u32 n_graphs;
    u32 single_gid;
    u32 max_n;             // largest graph of the launch (re-arm grid)
    u32 total_sources;
    LaunchCtl *ctl;
    u64 *stats;            // [worker_blocks][ST_COUNT]
    u64 *inj;              // injection queue slots
    u32 inj_mask;
    u32 nblocks;
    u64 *dq;               // per-block public deques, nblocks x (dq_mask+1)
    QCtr *dqc;
    u32 dq_mask;
    u32 smem_mask;
    u32 flags;
    u32 max_steal;
    u32 steal_policy;
    u32 node_cap;          // node pool size: a popped entry beyond it is a scheduler fault
    u32 idle_sleep_ns;     // wait of a non-thief idle warp
    u32 max_thieves;       // thief slots (blocks stealing / polling at once)
    u32 dq_stride;         // entries allocated per block deque (>= dq_mask + 1)
    u32 batch_max;         // activations a warp takes per step (1..32)
    u32 local_keep;        // shared-memory ring size above which new work goes public (0 = default)
    u32 thief_mode;        // 0 capped thief slots, 1 adaptive (parks and wake tickets)
    u32 has_modules;       // the launch's graphs compose other graphs (module tasks)
    u32 steal_backoff_ns;  // longest sleep of a thief whose round found nothing (0 = 512)
    u32 keep_idle;         // 1: the kept backlog grows with the block's idle warps
    u32 hand_batch;        // 1: a step's whole output (<= batch_max) stays with its warp while the ring is empty
    u32 *thief_slots;      // max_thieves words, each on its own 128-byte line
    u64 time_limit_ns;
    u64 *trace;            // TG_OPT_TRACE: per task {start ns, publish ns} (may be null)
    volatile u32 *cancel;  // host-mapped cancel flag (may be null)
    i32 *status_out;       // host-mapped per-gid statuses (may be null)
    // server mode
    const SubEntry *sub;   // submission ring (device memory), sub_mask + 1 entries
    u32 sub_mask;
    u32 comp_mask;
    volatile u64 *comp;    // completion ring (host-mapped): seq << 32 | status << 16 | gid
};

// Launch helpers implemented in tg_kernels.cu (all enqueue on `st`).
cudaError_t launch_rearm(const KParams &p, cudaStream_t st);
cudaError_t launch_module_rearm(const KParams &p, u32 gid, u32 n, cudaStream_t st);
cudaError_t launch_sched(const KParams &p, int blocks, int threads, cudaStream_t st, bool serve = false);
cudaError_t launch_finalize(const KParams &p, cudaStream_t st);
cudaError_t launch_clear(u64 *slots, size_t count, cudaStream_t st);
cudaError_t sched_occupancy(int threads, size_t dyn_smem, int *blocks_per_sm, bool serve = false);
size_t sched_dyn_smem(u32 smem_entries, u32 warps);
cudaError_t launch_bench_payload(u64 count, u32 rounds, u32 *checksum, cudaStream_t st);
cudaError_t launch_bench_payload_tasks(u32 n, const u32 *ids, const u32 *rounds, const u32 *cnt, u32 *checksum,
                                       cudaStream_t st);
cudaError_t launch_bench_atomics(u64 *words, u64 footprint, u64 count, u64 *sink, cudaStream_t st);
cudaError_t launch_bench_chain(u32 hops, u32 rounds, u32 *last, cudaStream_t st);
// Fresh records for an instance: the immutable half of the template's records
// at src_off (successor range, degrees, kind, parameters, id), join word =
// strong in-degree, count = digest = 0, written at dst_off (may equal src_off).
cudaError_t launch_instance_rearm(NodeSlot *slots, u64 src_off, u64 dst_off, u32 n, cudaStream_t st);
// Launch, once and with no work, every kernel the host may launch while the
// resident server runs, so that none of them is loaded for the first time
// then: with lazy module loading a first launch waits for the running
// kernel, which waits for that launch's work -- until its time limit.
cudaError_t preload_serving_kernels(cudaStream_t st);
cudaError_t launch_capture_task(NodeSlot *slots, u32 *outv, const u32 *edges, u32 u, u32 node_off, cudaStream_t st);
// tg_pack.cu: graph ingest, validation and CSR pack on the device.
// flags[PK_INVALID] / [PK_EDGE_KIND]: a cause of that status was found;
// flags[PK_NSRC]: sources; flags[PK_NCOND]: condition tasks.
enum { PK_INVALID = 0, PK_EDGE_KIND, PK_NSRC, PK_NCOND, PK_FLAGS };
struct PackBufs {          // device scratch, carved by pack_carve
    u8 *kinds, *weak;      // the copied inputs
    u32 *params, *src, *dst;
    u32 *k1, *v1;          // the sort's second buffers
    u32 *outdeg, *sin, *win, *is_src, *off, *srcpos;
    u32 *flags, *hist, *sums;
};
struct PackDest {          // where the packed graph goes
    NodeSlot *slots;       // the graph's first record
    u32 *edges;            // its successor lists, then its sources
    u32 edge_base;         // global edge-pool index of edges[0]
    u32 *chunk_gid;        // its chunk-table entries
    u32 n_chunks, gid;
    GDesc *desc;
    u32 seed, node_off, n_src, exec_cap;
};
size_t pack_scratch_bytes(u32 n, u32 m);
void pack_carve(char *base, u32 n, u32 m, PackBufs &b);
// steps 1-3 (statuses and counts into flags); the inputs are in b
cudaError_t pack_validate(const PackBufs &b, u32 n, u32 m, bool weak, cudaStream_t st);
// steps 4-5, after a validation that found nothing
cudaError_t pack_build(const PackBufs &b, u32 n, u32 m, const PackDest &d, cudaStream_t st);
// tg_result.cu: pack the count and digest of tasks [node_off, node_off + n) into dst[0, n)
cudaError_t launch_result_gather(const NodeSlot *slots, u32 node_off, u32 n, u64 *dst, cudaStream_t st);

}  // namespace tg
