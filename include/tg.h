/*
 * tg.h -- C-ABI of the device-resident task-graph executor (libtg.so).
 *
 * A graph mixes static tasks and condition tasks (Taskflow paper, section
 * "Conditional Tasking").  Edges out of a condition task are WEAK, all other
 * edges are STRONG (section "Scheduling Condition Tasks").  Execution starts
 * at the tasks with zero strong and zero weak in-edges; a task runs when its
 * remaining strong dependencies reach zero; a condition task returns an index
 * into its successors, counted in the order the edges were inserted, and
 * control jumps straight to that successor without touching any join counter
 * (Algorithm 4, execute_task).  The whole run -- join counters, condition
 * dispatch, work stealing -- happens inside one persistent CUDA kernel.
 *
 * Task payloads (the paper leaves task callables to the user): every task
 * computes a deterministic 32-bit value
 *     x = P(id, iter, insum, rounds)
 * where id is the task's index in its graph, iter its own prior execution
 * count, insum the 32-bit sum of the outputs delivered to this activation
 * (each strong predecessor delivers its output when it releases the edge, a
 * condition delivers its output to the successor it selects, a source gets
 * 0) and rounds comes from the task's parameter word.  Per task the library
 * keeps out (last x), cnt (executions) and dig (dig = mix(dig ^ x) per
 * execution, from 0).
 *
 * Conventions for every entry point
 *   - Returns a status int: TG_OK (0), TG_PENDING (1, tg_poll only) or a
 *     negative TG_ERR_*.  Nothing is thrown across the ABI.
 *   - Host input arrays are read during the call and never retained: the
 *     caller keeps ownership.
 *   - The device arena and the CUDA stream given to tg_ctx_create belong to
 *     the caller (e.g. a torch uint8 tensor and torch.cuda.Stream.cuda_stream)
 *     and must outlive the context.  The library sub-allocates the arena and
 *     never calls cudaMalloc for graph data.
 *   - tg_ctx / tg_graph / tg_batch handles are owned by the library until the
 *     matching destroy call.  Calls on one context must not be made
 *     concurrently from several host threads.
 *   - All device work is enqueued on the context's stream.
 */
#ifndef TG_H
#define TG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tg_ctx tg_ctx;
typedef struct tg_graph tg_graph;
typedef struct tg_batch tg_batch;

/* Task kinds (Conditional Tasking).  Parameter word of every task:
 *   bits 0-15  rounds of the payload's mixing loop
 *   bits 16-23 trip count T of a TG_COND_LOOP (1..255)
 *   bits 24-31 signed 8-bit return value of a TG_COND_CONST
 * Condition return values (iter = the condition's own prior executions,
 * nsucc = its out-degree, HC = seeded hash of (graph seed, id, iter)):
 *   TG_COND_BRANCH  HC mod nsucc
 *   TG_COND_LOOP    0 (loop back) unless (iter+1) mod T == 0, then the exit
 *                   index: 1 if nsucc <= 2, else 1 + HC mod (nsucc-1)
 *   TG_COND_CONST   the constant; an index outside [0, nsucc) schedules
 *                   nothing (that control path ends).
 * TG_MODULE (Composable Tasking; graphs made with tg_graph_create_composed):
 * the task runs its payload, then the graph it composes runs to completion
 * -- that graph's sources take the module task's output as their input sum,
 * its tasks keep their counts and digests across entries within a run --
 * and only then are the module task's successors released (strong edges)
 * with its output.  Two module tasks must not use one graph at the same
 * time: entering a graph that is in use ends the caller with TG_ERR_RACE;
 * an error inside the composed graph becomes the caller's status.
 * TG_SUBFLOW (Dynamic Tasking, joined subflow): the task runs its payload,
 * then spawns a fresh copy of its template graph (every task at its initial
 * state), whose sources take the task's output as their input sum; when the
 * copy completes, the task's successors are released with its output plus
 * the sum (mod 2^32) of the outputs of every execution of a static task
 * without successors in the copy.  Each subflow task owns one copy, so
 * subflows of different tasks run concurrently.  With bit 24 of its
 * parameter word set the subflow is detached: the task's successors are
 * released at once with its output, the copy runs on its own, and the run
 * (or the composed graph holding the task) ends only when the copy has
 * ended too; running the task again while its copy still runs is a race. */
enum { TG_STATIC = 0, TG_COND_BRANCH = 1, TG_COND_LOOP = 2, TG_COND_CONST = 3, TG_MODULE = 4,
       TG_SUBFLOW = 5 };

enum {
    TG_OK = 0,
    TG_PENDING = 1,          /* tg_poll: the submission has not finished */
    TG_ERR_INVALID = -1,     /* bad argument, index out of range, limit exceeded */
    TG_ERR_NO_SOURCE = -2,   /* no task with zero strong and zero weak in-edges */
    TG_ERR_EDGE_KIND = -3,   /* explicit weak[] disagrees with the source task's kind */
    TG_ERR_BUDGET = -4,      /* graph does not fit the memory budget / pools */
    TG_ERR_RACE = -5,        /* a task was activated while already queued or running */
    TG_ERR_EXEC_LIMIT = -6,  /* more executions than the per-graph cap */
    TG_ERR_TIMEOUT = -7,     /* the device-side time limit expired */
    TG_ERR_CANCELLED = -8,   /* tg_cancel was called while the graph ran */
    TG_ERR_CUDA = -9,        /* a CUDA runtime call failed */
    TG_ERR_INTERNAL = -10,   /* a bounded device wait gave up (scheduler fault) */
    TG_ERR_BUSY = -11        /* the graph is already submitted and not finished */
};

/* Option flags. */
#define TG_OPT_NO_RACE_CHECK 0x1u   /* skip the per-activation in-flight check (launches whose
                                       graphs have no condition, module or subflow tasks skip it
                                       anyway: every task runs once, a race cannot occur) */
#define TG_OPT_TRACE 0x2u           /* TG_OPT_TRACE_TASKS plus per-phase cycle counts
                                       (tg_ctx_get_stats), which only the extended scheduler
                                       variant keeps: launches run in it, slower */
#define TG_OPT_TRACE_TASKS 0x4u     /* record, for every task, when it was taken from a queue,
                                       when its step ended and where it was taken from
                                       (tg_trace_copy), in single-graph and batch launches (not
                                       in the resident server); the launches keep their lean
                                       scheduler variants and cost about the same */

/* Context options; a zero field selects the default (in brackets). */
typedef struct {
    int32_t worker_blocks;     /* persistent blocks [SMs x resident blocks per SM] */
    int32_t warps_per_block;   /* worker warps per block [16] */
    int32_t deque_depth;       /* entries of each block's public deque, power of 2 [4096] */
    int32_t steal_policy;      /* 0 random victims, 1 neighbour ring [0] */
    int32_t max_steal;         /* victims tried per steal round [8] */
    int32_t smem_ring;         /* entries of each block's shared-memory ready ring, power of 2 [1024] */
    uint32_t flags;            /* TG_OPT_* */
    uint32_t idle_sleep_ns;    /* wait of an idle warp that is not its block's thief [256] */
    int32_t max_thieves;       /* blocks allowed to steal / poll at the same time [16] */
    int32_t batch_max;         /* activations a warp takes per step, 1..32 [32] */
    int32_t local_keep;        /* ready activations a block keeps in shared memory before the
                                  rest goes to its stealable deque, <= smem_ring [32] */
    int32_t thief_mode;        /* 0: at most max_thieves blocks steal at once; 1: adaptive
                                  (Alg. 3/6): while a block is active at least one block
                                  steals, a failed thief other than the last one parks, and
                                  the last thief to find work wakes one parked block.  The
                                  resident server always uses 0. [0] */
    uint64_t time_limit_ns;    /* device time limit per launch [10 s] */
    uint64_t exec_cap;         /* executions per graph before TG_ERR_EXEC_LIMIT [2^31] */
    uint64_t mem_budget_bytes; /* admission budget for graph memory [the node/edge pools] */
    uint64_t max_nodes;        /* node pool capacity [derived from the arena] */
    uint64_t max_edges;        /* edge pool capacity [derived from the arena] */
    uint32_t steal_backoff_ns; /* longest sleep of a thief between steal rounds that found
                                  nothing: it doubles from 256 ns up to this.  Short sleeps
                                  find spilled work sooner on wide graphs; long ones leave
                                  the memory system to the busy warps of a long chain
                                  (at most 1,000,000) [512] */
    int32_t keep_idle;         /* 1: while another block is hungry, a block keeps beyond
                                  local_keep as many ready activations as its idle warps can
                                  take at once, before any goes to its stealable deque;
                                  0: it keeps local_keep.  Read by single-graph launches of
                                  graphs with condition tasks (a compiled variant of its
                                  own); other launches ignore it [0] */
    int32_t hand_batch;        /* 1: a warp whose step made at most batch_max activations
                                  ready keeps them all for its own next step while its
                                  block's ring is empty; 0: it keeps at most 2 and publishes
                                  the rest [0] */
} tg_ctx_opts;

/* Create a context on the current CUDA device.
 *   dev_arena, arena_bytes  caller-owned device memory (256-byte aligned)
 *   cuda_stream             cudaStream_t the library enqueues on (NULL = legacy)
 *   opts                    may be NULL (all defaults)
 * Errors: TG_ERR_INVALID (NULL out, misaligned or too small arena),
 *         TG_ERR_CUDA. */
int tg_ctx_create(void *dev_arena, size_t arena_bytes, void *cuda_stream,
                  const tg_ctx_opts *opts, tg_ctx **out);
int tg_ctx_destroy(tg_ctx *ctx);

/* Ingest, validate and pack a graph, then copy it to the device (section
 * "Scheduling Condition Tasks" for the strong/weak rule; Algorithm 8 for the
 * source set).
 *   n_nodes, kinds[n], params[n]   tasks (kinds TG_*; params as above)
 *   n_edges, src[m], dst[m]        edges src[i] -> dst[i] in insertion order;
 *                                  duplicates allowed, counted per edge
 *   weak[m]                        NULL, or explicit edge kinds that must equal
 *                                  "source task is a condition"
 *   seed                           graph seed of the condition hash
 * Validation order: TG_ERR_INVALID (unknown kind, index >= n, a condition
 * without successors, loop trip 0, out-degree or strong in-degree > 65535,
 * n == 0), then TG_ERR_EDGE_KIND, then TG_ERR_NO_SOURCE; TG_ERR_BUDGET if
 * the pools cannot hold it.  Packing: successors in insertion order, 32-byte
 * node records, strong in-degree per task, the source list.  The upload uses
 * the context's side stream and is complete when the call returns; a graph
 * may be created while other graphs run on the context stream. */
int tg_graph_create(tg_ctx *ctx, uint32_t n_nodes, const uint8_t *kinds, const uint32_t *params,
                    uint32_t n_edges, const uint32_t *src, const uint32_t *dst,
                    const uint8_t *weak, uint32_t seed, tg_graph **out);
/* As tg_graph_create (same arguments, host pointers; same statuses in the
 * same order; the same packed graph), with ingest, validation and packing
 * done on the device (Task Graph Representation, and the successor order
 * that Algorithm 8's condition dispatch indexes): the inputs are copied to
 * the device -- from pinned memory asynchronously, from pageable memory
 * through the driver's staging -- then the degrees are counted, the limits
 * checked, the edges sorted stably by source task (insertion order within
 * each task) and the records, successor lists and source list written.
 * Graphs with module or subflow tasks are refused (TG_ERR_INVALID: they use
 * tg_graph_create_composed).  The context keeps device scratch of about
 * 29 bytes per task and 17 per edge, allocated on first use and grown when a
 * larger graph comes (TG_ERR_BUDGET if that allocation fails); it is freed
 * with the context.  Uses the side stream; complete when the call returns.
 * While the resident server runs, the packing kernels share the SMs with it
 * (its blocks leave part of each SM free for side-stream work).
 * tg_graph_get_info: pack_ns = device time of validation and packing,
 * upload_ns = device time of the input copies. */
int tg_graph_create_dev(tg_ctx *ctx, uint32_t n_nodes, const uint8_t *kinds, const uint32_t *params,
                        uint32_t n_edges, const uint32_t *src, const uint32_t *dst,
                        const uint8_t *weak, uint32_t seed, tg_graph **out);
/* As tg_graph_create, with module tasks (Composable Tasking, "composed_of")
 * and subflow tasks (Dynamic Tasking): modules[n_nodes] names, for every
 * TG_MODULE task, the graph it composes and, for every TG_SUBFLOW task, the
 * template of its subflow (NULL for every other task).  A composed graph or
 * template belongs to the same context and is not an instance; a composed
 * graph may itself compose others, a template holds neither module nor
 * subflow tasks.  Each subflow task gets its own copy of its template at
 * creation (an instance, counted against the memory budget, freed with the
 * graph).  A graph used this way cannot be destroyed while a graph using it
 * exists (TG_ERR_BUSY).  A graph with
 * module tasks runs with tg_run / tg_submit: each launch starts every graph
 * it composes (transitively) from its initial state, and afterwards
 * tg_result_copy on a composed graph reads its tasks' results.  Batches may
 * hold such graphs (each launch re-arms every graph their compositions
 * reach; two members composing one graph run into each other: a race);
 * instances, the resident server and tg_capture_run refuse them
 * (TG_ERR_INVALID).  TG_ERR_INVALID also for a module task
 * without a graph, a graph given for another kind, or a foreign graph. */
int tg_graph_create_composed(tg_ctx *ctx, uint32_t n_nodes, const uint8_t *kinds, const uint32_t *params,
                             uint32_t n_edges, const uint32_t *src, const uint32_t *dst,
                             const uint8_t *weak, uint32_t seed, tg_graph *const *modules, tg_graph **out);
/* TG_ERR_BUSY while instances of g exist, while it is served, composed by
 * another graph or held by a live batch. */
int tg_graph_destroy(tg_ctx *ctx, tg_graph *g);

typedef struct {
    uint32_t n_nodes, n_edges, n_sources, n_conditions;
    uint64_t device_bytes;     /* pool bytes held by the graph */
    uint64_t pack_ns;          /* host time of validation + packing */
    uint64_t upload_ns;        /* host time of the host-to-device copy */
} tg_graph_info;
int tg_graph_get_info(const tg_graph *g, tg_graph_info *info);

/* Run one graph: re-arm its state, launch the persistent scheduler on the
 * context stream and wait -- the paper's "executor.run(taskflow).wait()"
 * (Static Tasking).  Returns the graph's final status (TG_OK, or
 * TG_ERR_RACE / EXEC_LIMIT / TIMEOUT / CANCELLED / INTERNAL / CUDA). */
int tg_run(tg_ctx *ctx, tg_graph *g);

/* Asynchronous form: enqueue the run and return at once -- submit_graph of
 * Algorithm 8 (the tasks with zero strong and zero weak dependencies go to
 * the shared queue first; here the re-arm kernel places them in the
 * injection queue the scheduler's thieves read).  *ticket names the
 * submission for tg_poll / tg_wait (the paper's run() returns a future);
 * it stays valid until g is submitted again or destroyed (a new submission
 * of g releases g's earlier tickets).  TG_ERR_BUSY if g is still in flight
 * (a graph must not run twice at once, Composable Tasking). */
int tg_submit(tg_ctx *ctx, tg_graph *g, uint64_t *ticket);
/* Never blocks: TG_PENDING while the run is in flight, else its status (a
 * non-blocking look at the future's state). */
int tg_poll(tg_ctx *ctx, uint64_t ticket);
/* Blocks until the submission finished; returns its status (the future's
 * wait(), Static Tasking). */
int tg_wait(tg_ctx *ctx, uint64_t ticket);

/* Make another execution instance of graph g: its own task state, outputs
 * and graph slot, sharing g's packed successor lists (no host packing: a
 * small kernel on a side stream copies the immutable half of g's task
 * records and sets the fresh state).  Several instances of one
 * graph may run at the same time.  Destroy it with tg_graph_destroy; g cannot
 * be destroyed while it has instances (TG_ERR_BUSY).  TG_ERR_BUDGET if the
 * memory budget or the pools cannot hold it. */
int tg_instance_create(tg_ctx *ctx, tg_graph *g, tg_graph **out);

/* Serving (continuous batching; the paper's co-run experiments run many
 * task graphs on one executor at once): start a resident scheduler on the
 * context stream.  While it runs, tg_submit queues a graph (or instance)
 * through a device submission ring -- its task state is re-armed by a small
 * kernel on the side stream (loaded before the server starts, so that its
 * first launch never waits for the running server) and the resident kernel
 * injects its sources while other graphs are running
 * -- and tg_poll / tg_wait read the completion records the kernel posts to
 * host-mapped memory.  tg_run and batches return TG_ERR_BUSY meanwhile.
 * The server runs one block per SM, with the context's warps per block
 * halved until two such blocks would fit on an SM, so that the kernels
 * re-arming instances can run beside it.
 * time_limit_ns bounds the server's lifetime (0 = 60 s); a graph still in
 * flight at the limit ends with TG_ERR_TIMEOUT.  Admission by memory budget
 * is the caller's loop: tg_instance_create / tg_graph_create fail with
 * TG_ERR_BUDGET until finished graphs are destroyed. */
int tg_serve_start(tg_ctx *ctx, uint64_t time_limit_ns);
/* Stop the resident scheduler and wait for it; returns TG_OK or the code
 * that ended it (TG_ERR_TIMEOUT, TG_ERR_INTERNAL). */
int tg_serve_stop(tg_ctx *ctx);

/* Request loop over a running server (the paper's co-run experiments run
 * many task graphs at once on one executor; here they are admitted while
 * others run): request i arrives arrival_ns[i] after the call starts
 * (ascending) and asks for one execution of templates[which[i]].  It is
 * admitted as soon as an instance fits the memory budget and a graph slot is
 * free (FIFO otherwise), submitted while other requests run, and its
 * instance is destroyed the moment it finishes, freeing budget for waiting
 * requests.  Per request: latency_ns[i] = finish minus arrival on the host
 * clock, status[i].  *max_in_flight (nullable) receives the most requests on
 * the device at once.  keep (nullable, n entries) receives each finished
 * instance instead of destroying it -- every request's, or with keep_mask
 * (nullable) only those whose mask byte is non-zero, the others getting
 * NULL -- so that its per-task results can be read with tg_result_copy; the
 * caller destroys kept instances, whose memory counts against the budget
 * until then.  Returns TG_OK or the first request's error. */
int tg_serve_replay(tg_ctx *ctx, tg_graph *const *templates, uint32_t n_templates, const uint32_t *which,
                    const uint64_t *arrival_ns, uint32_t n_requests, uint64_t *latency_ns, int *status,
                    uint32_t *max_in_flight, tg_graph **keep, const uint8_t *keep_mask);

/* Ask the device to stop: running graphs end with TG_ERR_CANCELLED (the
 * workers poll a host-mapped flag; the flag is cleared at the next launch). */
int tg_cancel(tg_ctx *ctx);

/* Copy the per-task results of g's last run to host arrays of n entries
 * (any pointer may be NULL); total_execs = sum of cnt.  Waits for g's last
 * launch only (a graph submitted after g may run meanwhile; a graph that
 * other graphs compose waits for the context stream), and reads on the side
 * stream through a device buffer of 8 bytes per task that the context
 * allocates on first use (TG_ERR_BUDGET if it cannot); while the resident
 * server runs, the records are read directly.  (The paper's tasks keep their results in user data; here
 * every task's last output, execution count and digest stay in the graph's
 * device state until its next run.)  Results are read by graph, not by
 * ticket: a graph holds the state of its last run, while a ticket only
 * names a submission.  A served request runs on an instance that the request
 * loop destroys when it finishes, freeing its memory for waiting requests;
 * to read a served request's results, keep its instance (tg_serve_replay's
 * keep / keep_mask) and pass that instance here. */
int tg_result_copy(tg_ctx *ctx, const tg_graph *g, uint32_t *out, uint32_t *cnt, uint32_t *dig,
                   uint64_t *total_execs);

/* Batches: many graphs in ONE persistent launch.  tg_batch_create writes the
 * launch's descriptor table and captures re-arm + scheduler kernels in a CUDA
 * graph; tg_batch_launch replays it (async); tg_batch_wait waits and writes
 * one status per graph.  A graph may belong to several batches but must not
 * run in two launches at once. */
int tg_batch_create(tg_ctx *ctx, tg_graph *const *gs, uint32_t n, tg_batch **out);
int tg_batch_launch(tg_ctx *ctx, tg_batch *b);
int tg_batch_wait(tg_ctx *ctx, tg_batch *b, int *statuses);
int tg_batch_destroy(tg_ctx *ctx, tg_batch *b);
/* Autotune a batch (worker-block count, warps per block, deque depth, steal
 * policy, victims per steal round, thief slots, activations per warp step,
 * local backlog and whether idle warps extend it, how much of a step's
 * output its warp keeps, thief mode, a thief's longest sleep and an idle
 * warp's sleep): time its launch under
 * candidate geometries by coordinate descent, `trials` timed launches each,
 * keep the fastest and re-capture the batch with it.  With cache_path
 * non-NULL, a result cached for the same device and batch shape (graph,
 * task, edge and source counts) is reused without searching; a new result is
 * appended to the file.  The batch's graphs run during the search (their
 * results are those of the last run).  *chosen and *best_ns may be NULL.
 * TG_ERR_* of the first failing launch if a graph does not end TG_OK. */
int tg_batch_autotune(tg_ctx *ctx, tg_batch *b, uint32_t trials, const char *cache_path,
                      tg_ctx_opts *chosen, uint64_t *best_ns);

/* Autotune one graph's launch geometry (the batch knobs above) by timing real runs
 * of it: `trials` timed runs per candidate after one warm-up, coordinate
 * descent, the winner cached under the device and graph shape in
 * cache_path (NULL: no cache).  The graph keeps the chosen geometry for its
 * later tg_run / tg_submit launches.  *chosen / *best_ns (may be NULL)
 * receive it and its best device time.  Runs the graph several times: its
 * results afterwards are those of its last run.  TG_ERR_BUSY while serving;
 * a run's error status ends the search and is returned. */
int tg_graph_autotune(tg_ctx *ctx, tg_graph *g, uint32_t trials, const char *cache_path, tg_ctx_opts *chosen,
                      uint64_t *best_ns);

/* Convenience: create, launch, wait and destroy; statuses may be NULL.
 * Returns TG_OK if every graph ended TG_OK, else the first error.  (The
 * paper runs several task graphs on one executor at once, co-run
 * experiments of Micro-benchmarks; here they share one persistent launch.) */
int tg_run_batch(tg_ctx *ctx, tg_graph *const *gs, uint32_t n, int *statuses);

/* Scheduler counters of the context's last launch (summed over blocks). */
typedef struct {
    uint64_t tasks;            /* activations executed */
    uint64_t pops_local;       /* batches taken from a block's shared-memory ring */
    uint64_t pops_own;         /* batches taken from the block's own public deque */
    uint64_t steal_attempts;   /* victim deques probed */
    uint64_t steal_hits;       /* probes that returned work */
    uint64_t inject_pops;      /* batches taken from the shared injection queue */
    uint64_t spills;           /* batches moved from shared memory to a public deque */
    uint64_t idle_loops;       /* warp iterations that found no work */
    uint64_t warp_iters;       /* warp iterations that executed work */
    uint64_t pops_hand;        /* batches a warp kept from its own previous step */
    uint64_t kernel_ns;        /* device time of the last scheduler launch */
    uint32_t worker_blocks, warps_per_block;
    uint64_t phase_cycles[5];  /* TG_OPT_TRACE only: SM cycles of the steps that executed work,
                                  split into taking the work, reading the task records, the
                                  payloads, the releases (with their race checks), and the
                                  flag release / publication / pending-count settle */
    uint64_t parks;            /* thief_mode 1: times a failed thief parked its block */
    uint64_t peak_thieves;     /* most blocks stealing at the same time (thief_mode 1) */
    uint64_t failed_rounds;    /* steal rounds (own deque, advertised victims, injection
                                  queue) that found nothing: the polling a thief policy wastes */
    uint64_t round_cycles;     /* SM cycles those failed rounds took (e_s of the paper's bound
                                  on wasteful steals = round_cycles / failed_rounds) */
} tg_stats;
int tg_ctx_get_stats(tg_ctx *ctx, tg_stats *st);
int tg_ctx_get_opts(const tg_ctx *ctx, tg_ctx_opts *opts);
/* Change the launch geometry used by later single-graph launches and by
 * batches created afterwards.  Reads worker_blocks, warps_per_block,
 * deque_depth (at most the context's), steal_policy, max_steal, smem_ring,
 * idle_sleep_ns, max_thieves, batch_max, local_keep, thief_mode,
 * steal_backoff_ns, keep_idle and hand_batch (0 = default); other fields are
 * ignored.
 * TG_ERR_INVALID if a field is out of range or the block shape cannot be
 * resident. */
int tg_ctx_set_launch(tg_ctx *ctx, const tg_ctx_opts *launch);

/* Roofline kernels (measurement only).
 *  tg_bench_payload: the task payload alone on `count` independent ids with
 *    `rounds` rounds each (no scheduling); *ns = device time; *checksum =
 *    XOR of all outputs (to compare with the oracle's payload).
 *  tg_bench_atomics: `count` returning 64-bit atomicAdd at distinct
 *    pseudo-random addresses over `footprint_words` 8-byte words of arena
 *    scratch; *ns = device time.
 *  tg_bench_chain: the dependency floor of a graph whose longest path has
 *    `hops` tasks of `rounds` rounds: one thread runs `hops` payloads in a
 *    row, each taking the previous output as its input sum (no scheduling);
 *    *ns = device time, *last = the final output. */
int tg_bench_payload(tg_ctx *ctx, uint64_t count, uint32_t rounds, uint64_t *ns, uint32_t *checksum);
int tg_bench_atomics(tg_ctx *ctx, uint64_t count, uint64_t footprint_words, uint64_t *ns);
/*  tg_bench_payload_tasks: the payload alone over a given multiset of
 *    executions (device arrays of n entries): task i runs cnt[i] payloads,
 *    iterations 0..cnt[i]-1, of rounds[i] rounds on id ids[i], one thread
 *    per task, so the arrays' order decides which executions share a warp;
 *    *ns = device time, *checksum = XOR of all outputs. */
int tg_bench_payload_tasks(tg_ctx *ctx, uint32_t n, const uint32_t *ids, const uint32_t *rounds,
                           const uint32_t *cnt, uint64_t *ns, uint32_t *checksum);
int tg_bench_chain(tg_ctx *ctx, uint32_t hops, uint32_t rounds, uint64_t *ns, uint32_t *last);

/* Capturer baseline (Algorithm 1): a static DAG as one kernel per task,
 * captured into a CUDA graph over round-robin streams.
 *  tg_levelize: host only.  level[v] = 0 for a task without in-edges, else
 *    1 + the largest level of its predecessors; index[v] = the task's
 *    position among the tasks of its level taken in ascending id.
 *    *n_levels = levels.  TG_ERR_INVALID for a bad index or a cycle.
 *  tg_stream_plan: host only.  stream[v] = index[v] mod max_streams
 *    (1..32); *n_events = tasks that record an event because a successor
 *    sits on another stream; *n_waits = distinct (predecessor, task) pairs
 *    on different streams, each a stream wait.
 *  tg_capture_run: run graph g (static tasks only, a DAG of at most 65,536
 *    tasks) as the CUDA graph Algorithm 1 builds with max_streams streams:
 *    a re-arm, then per task (level by level) one kernel on its stream that
 *    reads its input sum from its join word, runs the payload, writes its
 *    output, count and digest, and adds its output to each successor's join
 *    word; cross-stream edges become event waits.  Built on the first call
 *    per (g, max_streams), replayed afterwards; *ns = device time of the
 *    replay.  Results are read with tg_result_copy.  TG_ERR_INVALID for a
 *    condition task, a cycle, more than 65,536 tasks or max_streams outside
 *    1..32; TG_ERR_BUSY while g is in flight or the context serves. */
int tg_levelize(uint32_t n, uint32_t m, const uint32_t *src, const uint32_t *dst, uint32_t *level,
                uint32_t *index, uint32_t *n_levels);
int tg_stream_plan(uint32_t n, uint32_t m, const uint32_t *src, const uint32_t *dst, uint32_t max_streams,
                   uint32_t *stream, uint32_t *n_events, uint32_t *n_waits);
int tg_capture_run(tg_ctx *ctx, tg_graph *g, uint32_t max_streams, uint64_t *ns);

/* Run one graph without allocating anything (the paper has no counterpart:
 * this exists for callers that cannot allocate device memory, e.g. code
 * inside another framework's memory pool or a plugin handed fixed buffers).
 * All scratch memory lives in one fixed-size array inside the library that
 * every GPU loading the library holds until the process exits; no cudaMalloc,
 * cudaFree or other allocating routine is called.
 *   kinds[n], params[n]       device arrays, as for tg_graph_create
 *   succ_off[n+1], succ[m]    device arrays: task v's successors, in insertion
 *                             order, are succ[succ_off[v] .. succ_off[v+1])
 *   out[n], cnt[n], dig[n]    device outputs (any may be NULL)
 *   cuda_stream               stream the work is enqueued on; the call
 *                             synchronises it before returning
 * Limits: n <= 65536 tasks and m <= 262144 edges, else TG_ERR_BUDGET; the
 * scratch array is 6,892,032 bytes (about 6.6 MiB).
 * Returns the validation status (as tg_graph_create, checked on the device:
 * TG_ERR_INVALID also for a successor id >= n, succ_off decreasing or past
 * n_edges, or succ_off[n] != n_edges) or the run's status.
 * Every call shares the one scratch array: calls that overlap on the GPU
 * race.  The first call on a device sets that device up (looks up the
 * array's address).  The call cannot be made while cuda_stream is being
 * captured into a CUDA graph: it synchronises the stream and reads status
 * words back to the host. */
int tg_run_noalloc(uint32_t n_nodes, const uint8_t *kinds, const uint32_t *params,
                   const uint32_t *succ_off, const uint32_t *succ, uint32_t n_edges, uint32_t seed,
                   uint32_t *out, uint32_t *cnt, uint32_t *dig, void *cuda_stream);

/* Where a traced task was taken from (high half of a tg_trace_copy `where`
 * word; the low half is the worker block): */
#define TG_TRACE_FROM_HAND 0u        /* kept by the warp whose step made it ready */
#define TG_TRACE_FROM_RING 1u        /* the block's shared-memory ring */
#define TG_TRACE_FROM_OWN_DEQUE 2u   /* the block's own public deque */
#define TG_TRACE_FROM_STEAL 3u       /* another block's public deque */
#define TG_TRACE_FROM_INJECTION 4u   /* the shared injection queue (sources) */
/* With TG_OPT_TRACE_TASKS or TG_OPT_TRACE: for each of g's n tasks, its last
 * execution's device clock (ns, %globaltimer) when a warp took it from a
 * queue (start_ns) and when that warp's step ended, before the step's new
 * activations were published (end_ns), and where it was taken from (where =
 * TG_TRACE_FROM_* << 16 | worker block).  Any pointer may be NULL.  A task
 * that never ran reads 0.  TG_ERR_INVALID without either option. */
int tg_trace_copy(tg_ctx *ctx, const tg_graph *g, uint64_t *start_ns, uint64_t *end_ns, uint32_t *where);

/* The packed form of g as Graphviz DOT text: one node per task ("<id> <kind>
 * R=<rounds>", with the trip or constant of a condition and the composed
 * graph of a module or subflow task) and its edges in insertion order --
 * strong edges solid, weak edges dashed and labelled with their successor
 * index.  Read back from the device, so it shows what the scheduler runs.
 * *len receives the text's length (without the terminating NUL); the text is
 * written only if buf holds len + 1 bytes, else TG_ERR_BUDGET. */
int tg_graph_dot(tg_ctx *ctx, const tg_graph *g, char *buf, size_t cap, size_t *len);
/* The packed form of g word for word, as the device holds it (for tests and
 * debugging).  records[8 * n] receives each task's 32-byte record: successor
 * offset (relative to the graph's first successor entry), successor count |
 * strong in-degree << 16, rounds | kind << 16 | argument << 24, task id, join
 * word (low word first), execution count, digest.  edges receives the
 * graph's successor entries (graph-local ids; bit 31 marks a task's only
 * strong in-edge; a module or subflow task's list is led by a graph slot id)
 * followed by its source list; *edge_words (if not NULL) receives their
 * count.  Either array may be NULL.  Synchronises the context stream unless
 * the resident server runs. */
int tg_graph_packed_copy(tg_ctx *ctx, const tg_graph *g, uint32_t *records, uint32_t *edges,
                         uint64_t *edge_words);

const char *tg_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* TG_H */
