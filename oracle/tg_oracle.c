/*
 * tg_oracle.c -- the ORACLE: a plain, slow, sequential CPU executor of the
 * task-graph semantics.  Test infrastructure only: tests, the smoke check and
 * the benchmark's CPU-baseline leg may call it; the product path never does.
 * It shares no code, header or constant table with the CUDA path.
 *
 * What it follows (Huang et al., "Taskflow: A Lightweight Parallel and
 * Heterogeneous Task Graph Computing System"):
 *   - Task-level scheduling, "Scheduling Condition Tasks": an edge out of a
 *     condition task is weak, every other edge is strong; execution starts at
 *     the tasks with zero strong AND zero weak in-edges; a task runs when its
 *     remaining strong dependencies reach zero; a condition task skips that
 *     rule and jumps straight to the successor its return value indexes.
 *   - Conditional Tasking: the index refers to the successors in the order
 *     they were preceded (edge insertion order).
 *   - Algorithm 4 (execute_task): run the callable; a condition submits
 *     successors[r] and returns; any other task decrements every successor's
 *     strong counter and submits those that reach zero.
 *   - Algorithm 8 (submit_graph): the zero-dependency tasks are submitted first.
 *
 * Readings where the paper is silent (the same readings bind the CUDA path):
 *   - Join counters in cycles: the releaser that takes a counter to zero
 *     restores it to the strong in-degree (paper only decrements).
 *   - Out-of-range condition index: no successor is submitted.
 *   - A run ends when nothing is queued or running.
 *   - Task race ("only one thread can touch a task at a time"): an activation
 *     of a task that is already queued is reported as ORC_ERR_RACE.
 *   - The task callables are not in the paper.  Every task computes the
 *     payload P(id, iter, insum, rounds) below, where iter is the task's own
 *     prior execution count and insum is the sum (mod 2^32) of the outputs
 *     delivered to this activation: each strong predecessor delivers its
 *     output when it releases the edge, a condition delivers its output to the
 *     successor it selects, and a source's activation receives 0.
 *     Parity of the payload and hash definitions themselves is unpinned by
 *     the paper; they are pinned by invertibility of the mixing step, by the
 *     zero-round closed form and by frozen vectors.
 *
 * Build: gcc -O2 -shared -fPIC -o liboracle.so tg_oracle.c
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_STATIC = 0, ORC_COND_BRANCH = 1, ORC_COND_LOOP = 2, ORC_COND_CONST = 3 };
enum {
    ORC_OK = 0,
    ORC_ERR_INVALID = -1,
    ORC_ERR_NO_SOURCE = -2,
    ORC_ERR_EDGE_KIND = -3,
    ORC_ERR_RACE = -5,
    ORC_ERR_EXEC_LIMIT = -6,
    ORC_ERR_NOMEM = -10
};

/* "lowbias32" xorshift-multiply mixer (C. Wellons, "Prospecting for Hash
 * Functions", 2018; public domain).  A bijection of the 32-bit integers. */
uint32_t orc_mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

/* Task payload: a seed word made from (id, iter, insum), then `rounds`
 * rounds of "add the golden-ratio constant, mix". */
uint32_t orc_payload(uint32_t id, uint32_t iter, uint32_t insum, uint32_t rounds)
{
    uint32_t x = (id * 0x9E3779B9U) ^ (iter * 0x85EBCA6BU) ^ (insum * 0xC2B2AE35U) ^ 0x27D4EB2FU;
    for (uint32_t r = 0; r < rounds; ++r) {
        x += 0x9E3779B9U;
        x = orc_mix32(x);
    }
    return x;
}

/* Seeded condition hash of (graph seed, task id, task iteration). */
uint32_t orc_cond_hash(uint32_t seed, uint32_t id, uint32_t iter)
{
    return orc_mix32(orc_mix32(orc_mix32(seed ^ 0xA511E9B3U) ^ id) ^ iter);
}

/* The successor index a condition task returns (may be out of range).
 *   branch:   hash mod nsucc
 *   loop(T):  0 (back) unless (iter+1) is a multiple of T; then the exit
 *             index: 1 when nsucc <= 2, else 1 + hash mod (nsucc-1)
 *   constant: the signed 8-bit constant of the parameter word */
int32_t orc_condition_index(uint32_t kind, uint32_t param, uint32_t seed, uint32_t id,
                            uint32_t iter, uint32_t nsucc)
{
    if (kind == ORC_COND_BRANCH)
        return (int32_t)(orc_cond_hash(seed, id, iter) % nsucc);
    if (kind == ORC_COND_LOOP) {
        uint32_t trip = (param >> 16) & 0xFFu;
        if ((iter + 1u) % trip != 0u)
            return 0;
        if (nsucc <= 2u)
            return 1;
        return (int32_t)(1u + orc_cond_hash(seed, id, iter) % (nsucc - 1u));
    }
    return (int32_t)(int8_t)(uint8_t)(param >> 24);
}

/* Sequential executor.  Inputs: n tasks (kind, param), m edges (src[i] ->
 * dst[i]) in insertion order, optional explicit weak[] flags (must equal
 * "source task is a condition"), the graph seed and an execution cap.
 * Outputs (n entries each, caller-owned): last output, execution count and
 * digest of every task; *execs = total executions.  Returns ORC_OK or an
 * error; on an error detected before execution the outputs are untouched. */
int orc_run(uint32_t n, const uint8_t *kinds, const uint32_t *params, uint32_t m,
            const uint32_t *src, const uint32_t *dst, const uint8_t *weak, uint32_t seed,
            uint64_t exec_cap, uint32_t *out, uint32_t *cnt, uint32_t *dig, uint64_t *execs)
{
    /* --- validation ------------------------------------------------------ */
    for (uint32_t v = 0; v < n; ++v) {
        if (kinds[v] > ORC_COND_CONST)
            return ORC_ERR_INVALID;
        if (kinds[v] == ORC_COND_LOOP && ((params[v] >> 16) & 0xFFu) == 0u)
            return ORC_ERR_INVALID;
    }
    for (uint32_t e = 0; e < m; ++e)
        if (src[e] >= n || dst[e] >= n)
            return ORC_ERR_INVALID;

    uint32_t *outdeg = calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t *first = calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t *succ = malloc(((size_t)m + 1) * sizeof(uint32_t));
    uint32_t *fill = calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t *strong_in = calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t *weak_in = calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t *w_cnt = calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t *w_sum = calloc((size_t)n + 1, sizeof(uint32_t));
    uint8_t *queued = calloc((size_t)n + 1, 1);
    uint32_t *q_task = malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t *q_sum = malloc(((size_t)n + 1) * sizeof(uint32_t));
    int status = ORC_OK;
    if (!outdeg || !first || !succ || !fill || !strong_in || !weak_in || !w_cnt || !w_sum ||
        !queued || !q_task || !q_sum) {
        status = ORC_ERR_NOMEM;
        goto done;
    }

    /* successor lists in insertion order (counting sort by source, stable) */
    for (uint32_t e = 0; e < m; ++e)
        outdeg[src[e]]++;
    for (uint32_t v = 0, acc = 0; v < n; ++v) {
        first[v] = acc;
        acc += outdeg[v];
    }
    for (uint32_t e = 0; e < m; ++e)
        succ[first[src[e]] + fill[src[e]]++] = dst[e];

    for (uint32_t v = 0; v < n; ++v)
        if (kinds[v] != ORC_STATIC && outdeg[v] == 0) {
            status = ORC_ERR_INVALID;   /* a condition needs a successor to index */
            goto done;
        }
    for (uint32_t e = 0; e < m; ++e) {
        int is_weak = kinds[src[e]] != ORC_STATIC;   /* weak = out of a condition */
        if (weak && (weak[e] != 0) != is_weak) {
            status = ORC_ERR_EDGE_KIND;
            goto done;
        }
        if (is_weak)
            weak_in[dst[e]]++;
        else
            strong_in[dst[e]]++;
    }

    /* --- instance state ------------------------------------------------- */
    uint32_t n_src = 0;
    for (uint32_t v = 0; v < n; ++v) {
        w_cnt[v] = strong_in[v];
        w_sum[v] = 0;
        out[v] = cnt[v] = dig[v] = 0;
        if (strong_in[v] == 0 && weak_in[v] == 0)
            n_src++;
    }
    *execs = 0;
    if (n_src == 0) {
        status = ORC_ERR_NO_SOURCE;
        goto done;
    }

    /* FIFO of activations (task, insum); a task is queued at most once, so n
     * slots suffice.  Sources first, in ascending id order (Algorithm 8). */
    uint32_t head = 0, size = 0;
#define ORC_PUSH(task, sum)                                   \
    do {                                                      \
        uint32_t t_ = (task);                                 \
        if (queued[t_]) {                                     \
            status = ORC_ERR_RACE;                            \
            goto done;                                        \
        }                                                     \
        queued[t_] = 1;                                       \
        uint32_t at_ = head + size;                           \
        if (at_ >= n)                                         \
            at_ -= n;                                         \
        q_task[at_] = t_;                                     \
        q_sum[at_] = (sum);                                   \
        size++;                                               \
    } while (0)

    for (uint32_t v = 0; v < n; ++v)
        if (strong_in[v] == 0 && weak_in[v] == 0)
            ORC_PUSH(v, 0u);

    while (size > 0) {
        uint32_t v = q_task[head], s = q_sum[head];
        head = head + 1 == n ? 0 : head + 1;
        size--;
        queued[v] = 0;

        /* run the task (Algorithm 4, invoke_task_callable) */
        uint32_t iter = cnt[v];
        uint32_t x = orc_payload(v, iter, s, params[v] & 0xFFFFu);
        out[v] = x;
        cnt[v] = iter + 1;
        dig[v] = orc_mix32(dig[v] ^ x);
        if (++*execs > exec_cap) {
            status = ORC_ERR_EXEC_LIMIT;
            goto done;
        }

        if (kinds[v] != ORC_STATIC) {
            /* condition: jump to successors[r]; no join counter is touched */
            int32_t r = orc_condition_index(kinds[v], params[v], seed, v, iter, outdeg[v]);
            if (r >= 0 && (uint32_t)r < outdeg[v])
                ORC_PUSH(succ[first[v] + (uint32_t)r], x);
        } else {
            /* static: release every successor in order */
            for (uint32_t k = 0; k < outdeg[v]; ++k) {
                uint32_t u = succ[first[v] + k];
                w_sum[u] += x;
                if (--w_cnt[u] == 0) {
                    uint32_t total = w_sum[u];
                    w_cnt[u] = strong_in[u];
                    w_sum[u] = 0;
                    ORC_PUSH(u, total);
                }
            }
        }
    }
#undef ORC_PUSH

done:
    free(outdeg);
    free(first);
    free(succ);
    free(fill);
    free(strong_in);
    free(weak_in);
    free(w_cnt);
    free(w_sum);
    free(queued);
    free(q_task);
    free(q_sum);
    return status;
}

/* Bulk helpers so tests can evaluate many payloads / condition indices in
 * one foreign call. */
void orc_payload_many(uint64_t count, const uint32_t *id, const uint32_t *iter, const uint32_t *insum,
                      const uint32_t *rounds, uint32_t *x)
{
    for (uint64_t i = 0; i < count; ++i)
        x[i] = orc_payload(id[i], iter[i], insum[i], rounds[i]);
}

void orc_mix32_many(uint64_t count, const uint32_t *in, uint32_t *outp)
{
    for (uint64_t i = 0; i < count; ++i)
        outp[i] = orc_mix32(in[i]);
}
