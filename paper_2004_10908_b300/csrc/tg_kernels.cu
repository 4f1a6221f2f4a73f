// tg_kernels.cu -- the device side of the task-graph executor (sm_103a).
//
// One persistent kernel runs every task of one or many graphs.  A worker is a
// warp: it takes up to 32 ready activations at a time (one per lane), runs
// their payloads, dispatches conditions (Algorithm 4: a condition submits
// successors[r] and touches no join counter) and releases the strong
// successors of static tasks with 64-bit atomics on their join words
// (Algorithm 4: decrement, submit at zero); a successor whose only strong
// in-edge this is needs no counter (the decrement would always reach zero)
// and is submitted directly.  Ready activations live in
//   - a per-block ring in shared memory (the worker's local queue, Alg. 5),
//   - a per-block public deque in global memory that other blocks steal
//     from (Alg. 6/7: random victims, at most max_steal probes a round),
//   - one shared injection queue that receives the sources (Alg. 8) and
//     overflow.
// All rings are multi-producer multi-consumer with monotonically increasing
// 32-bit tickets and an EMPTY marker per slot; every wait is bounded.
// Module tasks run another graph to completion and resume as a continuation
// (Composable Tasking); subflow tasks do the same on a fresh copy of a
// template (Dynamic Tasking).  The scheduler comes in five compiled
// variants: lean one-shot kernels for one graph, for one graph without
// condition tasks, and for batches, an extended one-shot kernel with the
// optional features (module and subflow tasks, adaptive thieves, tracing),
// and the resident server.
#include <mutex>

#include "tg_internal.h"
#include "../../include/tg.h"

namespace tg {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSpinLimit = 1 << 20;     // bounded waits on a slot (iterations)
constexpr int kCasTries = 256;
constexpr u32 kStage = 256;             // staged activations per warp (shared memory)
constexpr int kRelUnroll = 4;           // successor releases in flight per lane
constexpr u32 kPerLaneMax = 4;          // widest fan-out released lane by lane (one round)
constexpr u32 kHandMax = 2;             // narrowest step output kept by the warp itself

// ---------------------------------------------------------------------------
// arithmetic of the method (payload, condition hash, digest)
// ---------------------------------------------------------------------------
// lowbias32 mixer (C. Wellons, 2018): xor-shift / odd-multiply steps.
__device__ __forceinline__ u32 mix32(u32 x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Task payload: seed word from (id, iter, insum), then `rounds` x (add the
// golden-ratio constant, mix).
__device__ __forceinline__ u32 task_payload(u32 id, u32 iter, u32 insum, u32 rounds)
{
    u32 x = (id * 0x9E3779B9U) ^ (iter * 0x85EBCA6BU) ^ (insum * 0xC2B2AE35U) ^ 0x27D4EB2FU;
#pragma unroll 4
    for (u32 r = 0; r < rounds; ++r) {
        x += 0x9E3779B9U;
        x = mix32(x);
    }
    return x;
}

__device__ __forceinline__ u32 cond_hash(u32 seed, u32 id, u32 iter)
{
    return mix32(mix32(mix32(seed ^ 0xA511E9B3U) ^ id) ^ iter);
}

// Successor index returned by a condition task (may be out of range).
__device__ __forceinline__ int cond_index(u32 kind, u32 arg, u32 seed, u32 id, u32 iter, u32 nsucc)
{
    if (kind == TG_COND_BRANCH)
        return (int)(cond_hash(seed, id, iter) % nsucc);
    if (kind == TG_COND_LOOP) {
        if ((iter + 1u) % arg != 0u)
            return 0;
        if (nsucc <= 2u)
            return 1;
        return (int)(1u + cond_hash(seed, id, iter) % (nsucc - 1u));
    }
    return (int)(signed char)(unsigned char)arg;
}

// ---------------------------------------------------------------------------
// memory helpers
// ---------------------------------------------------------------------------
// Relaxed loads/stores at GPU scope (generic addresses: global or shared).
// C `volatile` would make them system-scope strong accesses, which take a
// far slower path when thousands of warps poll.
__device__ __forceinline__ u64 vld64(const u64 *p)
{
    u64 v;
    asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void vst64(u64 *p, u64 v)
{
    asm volatile("st.relaxed.gpu.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ u32 vld32(const u32 *p)
{
    u32 v;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ i32 vldi(const i32 *p) { return (i32)vld32((const u32 *)p); }
__device__ __forceinline__ void vst32(u32 *p, u32 v)
{
    asm volatile("st.relaxed.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ u64 globaltimer()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u32 lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Release/acquire fence at GPU scope: orders this thread's earlier writes
// (outputs, state, flag releases) before its later publishing writes.  A
// sequentially consistent fence is not needed and costs far more.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// The same at block scope: enough when the only readers of what follows are
// warps of this block (its shared-memory ring), and far cheaper.
__device__ __forceinline__ void fence_acq_rel_cta() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }

// Shared-memory forms of the ring accesses (block scope): the block's own
// ring is only ever touched by the block's warps.
__device__ __forceinline__ u32 sh_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ u32 lds32(const u32 *p)
{
    u32 v;
    asm volatile("ld.relaxed.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(sh_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ u64 lds64_acq(const u64 *p)
{
    u64 v;
    asm volatile("ld.acquire.cta.shared.u64 %0, [%1];" : "=l"(v) : "r"(sh_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ u64 lds64(const u64 *p)
{
    u64 v;
    asm volatile("ld.relaxed.cta.shared.u64 %0, [%1];" : "=l"(v) : "r"(sh_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void sts64(u64 *p, u64 v)
{
    asm volatile("st.relaxed.cta.shared.u64 [%0], %1;" ::"r"(sh_addr(p)), "l"(v) : "memory");
}
__device__ __forceinline__ u32 cas_s32(u32 *p, u32 cmp, u32 val)
{
    u32 old;
    asm volatile("atom.relaxed.cta.shared.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "r"(sh_addr(p)), "r"(cmp), "r"(val) : "memory");
    return old;
}
template <bool kLocal> __device__ __forceinline__ u32 rld32(const u32 *p) { return kLocal ? lds32(p) : vld32(p); }
template <bool kLocal> __device__ __forceinline__ u32 rcas32(u32 *p, u32 c, u32 v) { return kLocal ? cas_s32(p, c, v) : atomicCAS(p, c, v); }

// ---------------------------------------------------------------------------
// multi-producer multi-consumer rings (shared or global memory)
// ---------------------------------------------------------------------------
struct Ring {
    u32 *head;
    u32 *tail;
    u64 *slots;
    u32 mask;
};

// Warp-cooperative pop into lanes [0, k).  A thief takes half of what it
// sees (at least one); an owner takes up to 32.  A pop from the block's
// shared-memory ring (kLocal) reads each slot with block-scope acquire: its
// producer published it after a block-scope release fence.
template <bool kLocal = false>
__device__ __forceinline__ int ring_pop(const Ring &r, bool thief, int lane, u64 &e, int &err, int want = 32)
{
    u32 h = 0;
    int k = 0;
    if (lane == 0) {
        for (int t = 0; t < kCasTries; ++t) {
            u32 hh = rld32<kLocal>(r.head), tt = rld32<kLocal>(r.tail);
            int avail = (int)(tt - hh);
            if (avail <= 0)
                break;
            int kk = thief ? min(want, (avail + 1) >> 1) : min(want, avail);
            if (rcas32<kLocal>(r.head, hh, hh + (u32)kk) == hh) {
                h = hh;
                k = kk;
                break;
            }
        }
    }
    k = __shfl_sync(kFull, k, 0);
    h = __shfl_sync(kFull, h, 0);
    e = kEmpty;
    if (lane < k) {
        u64 *s = r.slots + ((h + (u32)lane) & r.mask);
        u64 v = kLocal ? lds64_acq(s) : vld64(s);
        int spins = 0;
        while ((u32)v == kEmpty32) {   // reserved by its producer, not yet written
            if (++spins > kSpinLimit) {
                err = 1;
                break;
            }
            v = kLocal ? lds64_acq(s) : vld64(s);
        }
        if ((u32)v != kEmpty32) {
            if (kLocal)
                sts64(s, kEmpty);
            else
                vst64(s, kEmpty);
        }
        e = v;
    }
    return k;
}

// Warp-cooperative push of the lanes with `has`; all or nothing.
template <bool kLocal = false>
__device__ __forceinline__ bool ring_push(const Ring &r, bool has, u64 ent, int lane, int &err)
{
    u32 m = __ballot_sync(kFull, has);
    if (m == 0)
        return true;
    int k = __popc(m);
    u32 t = 0;
    int ok = 0;
    if (lane == 0) {
        for (int tr = 0; tr < kCasTries; ++tr) {
            u32 tt = rld32<kLocal>(r.tail), hh = rld32<kLocal>(r.head);
            if ((int)(tt + (u32)k - hh) > (int)(r.mask + 1u))
                break;   // full
            if (rcas32<kLocal>(r.tail, tt, tt + (u32)k) == tt) {
                t = tt;
                ok = 1;
                break;
            }
        }
    }
    ok = __shfl_sync(kFull, ok, 0);
    if (!ok)
        return false;
    t = __shfl_sync(kFull, t, 0);
    if (has) {
        u64 *s = r.slots + ((t + (u32)__popc(m & lanemask_lt(lane))) & r.mask);
        int spins = 0;
        while ((u32)(kLocal ? lds64(s) : vld64(s)) != kEmpty32) {   // previous occupant not yet taken
            if (++spins > kSpinLimit) {
                err = 1;
                break;
            }
        }
        if (kLocal)
            sts64(s, ent);
        else
            vst64(s, ent);
    }
    return true;
}

template <bool kLocal = false>
__device__ __forceinline__ u32 ring_size(const Ring &r) { return rld32<kLocal>(r.tail) - rld32<kLocal>(r.head); }

// ---------------------------------------------------------------------------
// the persistent scheduler
// ---------------------------------------------------------------------------
struct WarpCtx {
    Ring local;      // block's shared-memory ring
    Ring own;        // block's public deque
    Ring inj;        // shared injection queue
    u32 high_water;  // local ring size above which new work goes public while a block is hungry
    u32 keep_hi;     // local ring size above which new work always goes public
    const u32 *busy; // keep_idle launches: the block's warps executing work (shared memory)
    u32 nwarps;      // the block's warps
    u32 bmax;        // activations a warp takes per step
    const u32 *hungry;  // blocks whose thief found no work anywhere
    u32 hungry_v;       // lane 0: its value, loaded at the start of the warp's step
    u32 *avail_word; // this block's word / bit in the work-available bitmap
    u32 avail_bit;
    int err;
};

// The backlog a block keeps while another block is hungry: local_keep, and
// with keep_idle as much as its idle warps can take at once (a backlog that
// they start at once would only wait for a thief in a public deque).  kIdle:
// compiled in, in a variant of its own (the extra code alone cost the other
// variants 2-6 % per hop).
template <bool kIdle>
__device__ __forceinline__ u32 local_limit(const WarpCtx &w)
{
    if (!kIdle || !w.busy)
        return w.high_water;
    const u32 idle = w.nwarps - min(lds32(w.busy), w.nwarps);
    return max(w.high_water, idle * w.bmax);
}

// Route the new ready activations of the warp (lanes with `has`).
template <bool kIdle = false>
__device__ __forceinline__ void emit(WarpCtx &w, bool has, u64 ent, int lane, u32 &spill_ctr, u64 *pe_order = nullptr)
{
    if (__ballot_sync(kFull, has) == 0)
        return;
    // spill beyond a short backlog while some block is idle, beyond a long
    // one otherwise (the hungry count was loaded when the step began, so
    // its latency is not on the publication path)
    int spill = 0;
    if (lane == 0) {
        const u32 lsz = ring_size<true>(w.local);
        spill = lsz >= w.keep_hi || (lsz >= local_limit<kIdle>(w) && (i32)w.hungry_v > 0);
    }
    spill = __shfl_sync(kFull, spill, 0);
    bool pub = has && spill;
    bool loc = has && !pub;
    if (!ring_push<true>(w.local, loc, ent, lane, w.err))
        pub = pub || loc;
    if (__ballot_sync(kFull, pub) != 0) {
        // work leaving the block: what precedes it is made visible GPU-wide
        // (the block's own ring needed only a block-scope fence).  An acyclic
        // launch of one graph (pe_order: its pending-count word) has only the
        // step's pending-count reservation to order, since nothing reads a
        // task's stored state while it runs: a returning no-op atomic on the
        // same word is performed after the reservation (same thread, same
        // address), and lane 0 takes the deque slots only once it returned.
        // A GPU-scope fence here waited for every outstanding store of the
        // warp, about 1.7 us at the median, on the path of stolen tasks.
        if (pe_order) {
            if (lane == 0 && atomicAdd(pe_order, 0ull) == kEmpty)
                w.err = 5;   // (never: the word's high half counts executions)
        } else {
            fence_acq_rel_gpu();
        }
        if (lane == 0)
            spill_ctr++;
        if (ring_push(w.own, pub, ent, lane, w.err)) {
            if (lane == 0 && (vld32(w.avail_word) & w.avail_bit) == 0u)
                atomicOr(w.avail_word, w.avail_bit);
        } else if (!ring_push(w.inj, pub, ent, lane, w.err)) {
            w.err = 2;
        }
    }
}

// Examine the result of the previous iteration's pending-count update: a
// graph whose pending count reached zero is complete; one whose execution
// count passed its cap is poisoned with TG_ERR_EXEC_LIMIT.
template <bool kServe, bool kExt>
__device__ __forceinline__ u64 settle_finish(const KParams &p, bool &pend, u64 old, u64 delta, u32 g, u32 cap)
{
    if (!pend)
        return kEmpty;
    u64 cont = kEmpty;
    const u64 nw = old + delta;
    if ((u32)(nw >> 32) > cap)
        atomicCAS(&p.descs[g].status, 0, TG_ERR_EXEC_LIMIT);
    if ((u32)nw == 0u) {
        u32 ret = (!kServe && kExt) ? vld32(&p.descs[g].ret) : kEmpty32;
        // a detached subflow's copy is done: it gives back its token of the
        // parent graph's pending count, which may complete the parent in turn
        // (bounded: a template holds no subflow tasks, so one level at most)
        for (int hop = 0; !kServe && kExt && ret != kEmpty32 && (ret & kDetachBit) != 0u && hop < 2; ++hop) {
            const u32 parent = __ldg(&p.chunk_gid[(ret & ~kDetachBit) >> kChunkShift]);
            const i32 st = vldi(&p.descs[g].status);
            if (st != 0)
                atomicCAS(&p.descs[parent].status, 0, st);
            vst32(&p.descs[g].ret, kEmpty32);
            fence_acq_rel_gpu();
            const u64 was = atomicAdd(&p.descs[parent].pe, ~0ull);   // - 1
            if ((u32)was != 1u) {
                ret = kEmpty32;
                g = kEmpty32;   // the parent still runs: nothing completes here
                break;
            }
            g = parent;
            ret = vld32(&p.descs[g].ret);
        }
        if (g == kEmpty32) {
            // done above
        } else if (ret != kEmpty32) {
            // a composed graph is done: its module task resumes (a
            // continuation activation) and inherits its status
            const i32 st = vldi(&p.descs[g].status);
            if (st != 0)
                atomicCAS(&p.descs[__ldg(&p.chunk_gid[ret >> kChunkShift])].status, 0, st);
            vst32(&p.descs[g].ret, kEmpty32);
            cont = (u64)ret;
        } else if (kServe) {
            // the graph is done: post a completion record to the host
            fence_acq_rel_gpu();
            const i32 st = vldi(&p.descs[g].status);
            const u32 idx = atomicAdd(&p.ctl->comp_tail, 1u);
            p.comp[idx & p.comp_mask] = ((u64)(idx + 1u) << 32) | ((u64)((u32)st & 0xFFFFu) << 16) | (u64)(g & 0xFFFFu);
            __threadfence_system();
        } else {
            atomicSub(&p.ctl->graphs_left, 1u);
        }
    }
    pend = false;
    return cont;
}

// A load that stays where it is written (the compiler may not sink it
// towards its first use): issued before the payload, its latency hides
// under it.  Predicated: with `pred` false nothing is read and 0 returned.
template <bool kServe>
__device__ __forceinline__ u32 ld_early(const u32 *ptr, bool pred)
{
    u32 v = 0;
    if (kServe)
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.cg.u32 %0, [%1];\n\t}"
                     : "+r"(v) : "l"(ptr), "r"((u32)pred));
    else
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.u32 %0, [%1];\n\t}"
                     : "+r"(v) : "l"(ptr), "r"((u32)pred));
    return v;
}

// Loads of data that is immutable while its graph exists: through L1 for a
// one-shot launch; through L2 for the resident server, whose node ranges and
// graph slots are recycled while it runs.
template <bool kServe, typename T>
__device__ __forceinline__ T ld_imm(const T *ptr)
{
    if (kServe)
        return __ldcg(ptr);
    return __ldg(ptr);
}

// Stage the new activations of the lanes with `has` in the warp's buffer;
// a full buffer is published early (its owners keep their flags meanwhile).
__device__ __forceinline__ void stage(WarpCtx &w, u64 *buf, u32 &ns, bool has, u64 ent, int lane, u32 &spill_ctr,
                                      u64 *pe_resv = nullptr)
{
    const u32 m = __ballot_sync(kFull, has);
    if (m == 0)
        return;
    const u32 k = (u32)__popc(m);
    if (ns + k > kStage) {
        // pe_resv: the activations are reserved here, as they leave the warp
        if (pe_resv && lane == 0)
            atomicAdd(pe_resv, (u64)ns);
        fence_acq_rel_cta();   // the pending-count reservation first
        __syncwarp();
        for (u32 i = 0; i < ns; i += 32u) {
            const bool h = i + (u32)lane < ns;
            emit(w, h, h ? buf[i + lane] : 0ull, lane, spill_ctr, pe_resv);
        }
        ns = 0;
        __syncwarp();
    }
    if (has)
        buf[ns + (u32)__popc(m & lanemask_lt(lane))] = ent;
    ns += k;
}

template <bool kIdle = false>
__device__ __forceinline__ void publish(WarpCtx &w, u64 *buf, u32 ns, int lane, u32 &spill_ctr, u64 *pe_order = nullptr)
{
    __syncwarp();
    u32 done = 0;
    if (ns > 32u) {
        // one reservation of the block ring's slots for the batches that the
        // per-batch rule in emit would keep local (a batch of 32 stays in the
        // block while the ring holds fewer than the backlog limit), instead of
        // one reservation per batch of 32 after the previous batch's
        u32 t = 0, nl = 0;
        if (lane == 0) {
            for (int tr = 0; tr < kCasTries; ++tr) {
                const u32 tt = lds32(w.local.tail), hh = lds32(w.local.head);
                const u32 lsz = tt - hh;
                const u32 thr = (i32)w.hungry_v > 0 ? min(local_limit<kIdle>(w), w.keep_hi) : w.keep_hi;
                u32 want = lsz < thr ? min(ns, ((thr - lsz + 31u) / 32u) * 32u) : 0u;
                want = min(want, (w.local.mask + 1u) - min(lsz, w.local.mask + 1u));
                if (want == 0u)
                    break;
                if (cas_s32(w.local.tail, tt, tt + want) == tt) {
                    t = tt;
                    nl = want;
                    break;
                }
            }
        }
        nl = __shfl_sync(kFull, nl, 0);
        t = __shfl_sync(kFull, t, 0);
        for (u32 j = (u32)lane; j < nl; j += 32u) {
            u64 *slot = w.local.slots + ((t + j) & w.local.mask);
            int spins = 0;
            while ((u32)lds64(slot) != kEmpty32) {   // previous occupant not yet taken
                if (++spins > kSpinLimit) {
                    w.err = 1;
                    break;
                }
            }
            sts64(slot, buf[j]);
        }
        done = nl;
    }
    for (u32 i = done; i < ns; i += 32u) {
        const bool h = i + (u32)lane < ns;
        emit<kIdle>(w, h, h ? buf[i + lane] : 0ull, lane, spill_ctr, pe_order);
    }
}

// The scheduler's body.  kExt: the launch uses an optional feature -- module
// or subflow tasks, the adaptive thief mode or tracing -- which lives in a
// separate variant, so that other launches carry none of that code (it costs
// them 5-19 % per dependency hop, measured).
template <bool kServe, bool kExt, bool kOne, bool kAcyc = false, bool kTrace = false, bool kIdle = false>
__device__ __forceinline__ void sched_body(const KParams &p)
{
    extern __shared__ u64 s_ring[];
    __shared__ u32 s_head, s_tail;
    __shared__ u32 s_push[32 * 32];
    __shared__ u32 s_keep[32 * 32];
    __shared__ u64 s_stats[ST_COUNT];
    __shared__ int s_thief, s_stop, s_hungry;
    __shared__ u32 s_busy, s_peak;
    __shared__ u64 s_tmark[32];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const u32 ring_n = p.smem_mask + 1u;
    for (u32 i = threadIdx.x; i < ring_n; i += blockDim.x)
        s_ring[i] = kEmpty;
    if (threadIdx.x < ST_COUNT)
        s_stats[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_head = 0;
        s_tail = 0;
        s_thief = 0;
        s_stop = 0;
        s_hungry = 0;
        s_busy = 0;
        s_peak = 0;
    }
    __syncthreads();

    // A launch whose graphs have no condition tasks (and compose nothing)
    // runs every task exactly once: no activation can find its target in
    // flight, so the in-flight flags -- one returning atomic per released
    // successor -- are skipped, and the task's own state is stored without a
    // fence of its own.
    // (kAcyc: the same known at compile time, every task is a static one)
    const bool acyclic = kAcyc || (!kServe && (p.flags & kFlagAcyclic) != 0u);

    const bool race_check = !acyclic && (p.flags & TG_OPT_NO_RACE_CHECK) == 0;
    const int bmax = (int)min(32u, max(1u, p.batch_max));
    // one graph: every activation has gid == single_gid (not when it composes others)
    // kOne: a lean launch of one graph (no launch table); every activation
    // then has gid == single_gid
    constexpr bool single = !kServe && !kExt && kOne;
    constexpr bool modules = !kServe && kExt;
    const u32 single_cap = single ? ld_imm<kServe>(&p.descs[p.single_gid].exec_cap) : 0u;
    const u64 t0 = globaltimer();
    const u64 deadline = t0 + p.time_limit_ns;

    WarpCtx w;
    w.local = Ring{&s_head, &s_tail, s_ring, p.smem_mask};
    w.own = Ring{&p.dqc[blockIdx.x].head, &p.dqc[blockIdx.x].tail,
                 p.dq + (size_t)blockIdx.x * p.dq_stride, p.dq_mask};
    w.inj = Ring{&p.ctl->inj.head, &p.ctl->inj.tail, p.inj, p.inj_mask};
    // a short shared-memory backlog while other blocks are idle (beyond it,
    // new activations go to the public deque where their thieves steal
    // them), half the ring while none is
    w.high_water = min(p.local_keep ? p.local_keep : 32u, ring_n);
    w.keep_hi = max(w.high_water, ring_n / 2u);
    w.busy = (kIdle && p.keep_idle) ? &s_busy : nullptr;
    w.nwarps = blockDim.x >> 5;
    w.bmax = (u32)bmax;
    w.hungry = &p.ctl->hungry;
    w.hungry_v = 0;
    w.err = 0;
    w.avail_word = &p.ctl->avail[blockIdx.x >> 5];
    w.avail_bit = 1u << (blockIdx.x & 31u);
    // a composed graph's completion resumes its module task: published after a fence
    auto resume = [&](u64 cont, u32 &spill_ctr) {
        if (!modules)
            return;
        const bool h = cont != kEmpty;
        if (__ballot_sync(kFull, h) != 0u) {
            fence_acq_rel_gpu();
            emit(w, h, cont, lane, spill_ctr);
        }
    };
    u32 *my_push = s_push + warp * 32;
    u32 *my_keep = s_keep + warp * 32;
    u64 *my_stage = s_ring + ring_n + (size_t)warp * kStage;

    // per-warp counters, 32-bit (registers are scarce); idle loops may exceed 2^32 in a long-lived server
    u32 st_tasks = 0, st_local = 0, st_own = 0, st_try = 0, st_hit = 0, st_inj = 0, st_spill = 0,
        st_iters = 0, st_hand = 0, st_park = 0, st_fail = 0;
    u64 st_idle = 0;
    u64 st_rcyc = 0, r_t0 = 0;   // SM cycles of the steal rounds that found nothing (lane 0)
    // adaptive thieves (Alg. 3/6 invariant): a block is active while one of
    // its warps executes; blocks are the workers whose counts are kept
    const bool adaptive = !kServe && kExt && p.thief_mode == 1u;
    // busy warps are counted for the adaptive thieves and for keep_idle
    const bool count_busy = adaptive || (kIdle && p.keep_idle != 0u);
    bool busy_w = false;
    u32 rng = mix32(blockIdx.x * 0x9E3779B9U + (u32)warp * 0x85EBCA6BU + 1u);
    bool pend = false;      // a pending-count update whose result is not examined yet
    u64 pend_old = 0, pend_delta = 0;
    u32 pend_g = 0, pend_cap = 0;
    u32 backoff = 256;
    const u32 backoff_max = p.steal_backoff_ns ? p.steal_backoff_ns : 512u;
    const u32 my_slot = blockIdx.x % p.max_thieves;
    u32 idle = 0;
    u32 noslot = 0;
    // activations this warp kept for itself (lanes [0, nh) of `hand`)
    u64 hand = kEmpty;
    int nh = 0;
    // kAcyc: the records of the kept activations, loaded when they were kept
    uint4 hand_imm = make_uint4(0u, 0u, 0u, 0u);
    bool hand_pre = false;
    // per-lane cache of the lane's graph descriptor; the status word is
    // re-read every 16 activations, so a poisoned graph drains soon after
    u32 c_gid = kEmpty32, c_seed = 0, c_cap = 0, c_age = 0, c_base = 0;
    i32 c_status = 0;

    // traced launches: cycles per phase of a step, marked by lane 0 (the
    // previous mark of each warp lives in shared memory)
    const bool traced = kExt && p.trace != nullptr && (p.flags & TG_OPT_TRACE) != 0u;
    // per-task records (TG_OPT_TRACE_TASKS or TG_OPT_TRACE), compiled only
    // into the extended and the traced variants: where this warp's current
    // activations were taken from
    const bool task_trace = (kExt || kTrace) && !kServe && p.trace != nullptr;
    u32 from = TG_TRACE_FROM_HAND;
    auto mark = [&](int phase) {
        if (traced && lane == 0) {
            const u64 t = clock64();
            if (phase >= 0)
                atomicAdd(&s_stats[ST_PHASE0 + phase], t - s_tmark[warp]);
            s_tmark[warp] = t;
        }
    };
    for (;;) {
        u64 e = kEmpty;
        int k = 0;
        mark(-1);
        bool pre_now = false;
        if (nh) {
            e = hand;
            k = nh;
            nh = 0;
            pre_now = hand_pre;
            st_hand++;
            from = TG_TRACE_FROM_HAND;
        } else {
            k = ring_pop<true>(w.local, false, lane, e, w.err, bmax);
            if (k) {
                st_local++;
                from = TG_TRACE_FROM_RING;
            } else {
                resume(settle_finish<kServe, kExt>(p, pend, pend_old, pend_delta, pend_g, pend_cap), st_spill);
                if (count_busy && busy_w) {
                    busy_w = false;
                    if (lane == 0 && atomicSub(&s_busy, 1u) == 1u && adaptive)
                        atomicSub(&p.ctl->actives, 1u);
                }
                // ---- idle.  One warp per block at a time is the block's thief
                // (Alg. 6/7), and at most max_thieves blocks steal at once; only
                // thieves poll launch-wide state, the other idle warps wait on
                // shared memory, so idle polling never floods L2.
                // leave together: a warp whose lanes split here would wait
                // forever in its next warp-wide operation
                if (__any_sync(kFull, *(volatile int *)&s_stop != 0))
                    break;
                int am = 0;
                if (lane == 0) {
                    am = atomicCAS(&s_thief, 0, 1) == 0;
                    if (am && adaptive) {
                        const u32 t = atomicAdd(&p.ctl->thieves, 1u) + 1u;
                        atomicMax(&s_peak, t);
                    } else if (am && atomicCAS(&p.thief_slots[my_slot * 32u], 0u, 1u) != 0u) {
                        *(volatile int *)&s_thief = 0;
                        am = 2;
                    }
                }
                am = __shfl_sync(kFull, am, 0);
                if (am != 1) {
                    st_idle++;
                    if (am == 2) {
                        // no thief slot: still notice the end of the launch, at a
                        // low rate (one read per block every few microseconds)
                        int stop = 0;
                        if (lane == 0 && ((++noslot & 3u) == 0u)) {
                            const bool done = kServe ? (vld32(&p.ctl->stop) != 0u) : (vld32(&p.ctl->graphs_left) == 0u);
                            if (done || vldi(&p.ctl->abort_code) != 0) {
                                stop = 1;
                            } else if (globaltimer() > deadline) {
                                atomicCAS(&p.ctl->abort_code, 0, TG_ERR_TIMEOUT);
                                stop = 1;
                            }
                            if (stop)
                                *(volatile int *)&s_stop = 1;
                        }
                        if (__shfl_sync(kFull, stop, 0))
                            break;
                    }
                    __nanosleep(am == 2 ? backoff : p.idle_sleep_ns);
                    if (am == 2)
                        backoff = min(backoff * 2u, backoff_max);
                    continue;
                }
                if (lane == 0)
                    r_t0 = clock64();
                if (kServe) {
                    // claim the next submitted graph, re-arm its pending
                    // count and status, and take its sources (Algorithm 8)
                    u32 cg = kEmpty32;
                    SubEntry subv{};
                    if (lane == 0) {
                        const u32 h = vld32(&p.ctl->sub_head);
                        const SubEntry *se = &p.sub[h & p.sub_mask];
                        if (vld32(&se->seq) == h + 1u && atomicCAS(&p.ctl->sub_head, h, h + 1u) == h) {
                            cg = vld32(&se->gid);
                            subv.node_off = vld32(&se->node_off);
                            subv.n = vld32(&se->n);
                            subv.seed = vld32(&se->seed);
                            subv.src_off = vld32(&se->src_off);
                            subv.n_src = vld32(&se->n_src);
                            subv.exec_cap = vld32(&se->exec_cap);
                        }
                    }
                    cg = __shfl_sync(kFull, cg, 0);
                    subv.node_off = __shfl_sync(kFull, subv.node_off, 0);
                    subv.n = __shfl_sync(kFull, subv.n, 0);
                    subv.seed = __shfl_sync(kFull, subv.seed, 0);
                    subv.src_off = __shfl_sync(kFull, subv.src_off, 0);
                    subv.n_src = __shfl_sync(kFull, subv.n_src, 0);
                    subv.exec_cap = __shfl_sync(kFull, subv.exec_cap, 0);
                    if (cg != kEmpty32) {
                        // the entry carries the graph's descriptor: write it and
                        // the graph's chunk-table entries, then its sources
                        GDesc &D = p.descs[cg];
                        const u32 base = subv.node_off;
                        const u32 n_src = subv.n_src;
                        const u32 src_off = subv.src_off;
                        if (lane == 0) {
                            vst32(&D.seed, subv.seed);
                            vst32(&D.node_off, base);
                            vst32(&D.n, subv.n);
                            vst32(&D.src_off, src_off);
                            vst32(&D.n_src, n_src);
                            vst32(&D.exec_cap, subv.exec_cap);
                            vst64(&D.pe, (u64)n_src);
                            vst32((u32 *)&D.status, 0u);
                        }
                        const u32 n_chunks = (subv.n + kChunk - 1u) >> kChunkShift;
                        for (u32 i = (u32)lane; i < n_chunks; i += 32u)
                            vst32(const_cast<u32 *>(&p.chunk_gid[(base >> kChunkShift) + i]), cg);
                        fence_acq_rel_gpu();
                        __syncwarp();
                        for (u32 i = 0; i < n_src; i += 32u) {
                            const bool h = i + (u32)lane < n_src;
                            const u64 ent = h ? (u64)(base + __ldcg(&p.edges[src_off + i + (u32)lane])) : 0ull;
                            emit(w, h, ent, lane, st_spill);
                        }
                        st_inj++;
                        from = TG_TRACE_FROM_INJECTION;
                        k = ring_pop<true>(w.local, false, lane, e, w.err, bmax);
                    }
                }
                if (k == 0)
                    k = ring_pop(w.own, false, lane, e, w.err, bmax);
                if (k) {
                    st_own++;
                    from = TG_TRACE_FROM_OWN_DEQUE;
                } else {
                    if (lane == 0 && (vld32(w.avail_word) & w.avail_bit) != 0u) {
                        atomicAnd(w.avail_word, ~w.avail_bit);
                        if (ring_size(w.own) != 0u)
                            atomicOr(w.avail_word, w.avail_bit);
                    }
                    // victims: blocks whose availability bit is set, scanned from
                    // a random (or, for the ring policy, the next) block
                    const u32 nwords = (p.nblocks + 31u) >> 5;
                    u32 word = (u32)lane < nwords ? vld32(&p.ctl->avail[lane]) : 0u;
                    if ((u32)lane == (blockIdx.x >> 5))
                        word &= ~(1u << (blockIdx.x & 31u));
                    const u32 nonempty = __ballot_sync(kFull, word != 0u);
                    u32 start;
                    if (p.steal_policy == 1) {
                        start = blockIdx.x + 1u;
                    } else {
                        rng = rng * 1664525u + 1013904223u;
                        start = (u32)(((unsigned long long)(rng >> 8) * p.nblocks) >> 24);
                    }
                    u32 tries = 0;
                    if (nonempty) {
                        for (u32 i = 0; i < nwords && k == 0 && tries < p.max_steal; ++i) {
                            const u32 wi = ((start >> 5) + i) % nwords;
                            u32 bits = __shfl_sync(kFull, word, (int)wi);
                            if (i == 0)
                                bits &= ~((1u << (start & 31u)) - 1u);
                            while (bits && k == 0 && tries < p.max_steal) {
                                const u32 v = wi * 32u + (u32)(__ffs(bits) - 1);
                                bits &= bits - 1u;
                                if (v >= p.nblocks)
                                    break;
                                Ring vr{&p.dqc[v].head, &p.dqc[v].tail, p.dq + (size_t)v * p.dq_stride,
                                        p.dq_mask};
                                st_try++;
                                tries++;
                                k = ring_pop(vr, true, lane, e, w.err, bmax);
                                if (k) {
                                    st_hit++;
                                    from = TG_TRACE_FROM_STEAL;
                                } else if (lane == 0) {
                                    // drained: clear the bit, then re-check so a
                                    // spill that raced with the clear stays visible
                                    atomicAnd(&p.ctl->avail[v >> 5], ~(1u << (v & 31u)));
                                    if (ring_size(vr) != 0u)
                                        atomicOr(&p.ctl->avail[v >> 5], 1u << (v & 31u));
                                }
                            }
                        }
                    }
                    if (k == 0) {
                        k = ring_pop(w.inj, true, lane, e, w.err, bmax);
                        if (k)
                            st_inj++;
                            from = TG_TRACE_FROM_INJECTION;
                    }
                }
                if (k == 0) {
                    // stop when every graph is done, on abort, timeout or cancel
                    st_idle++;
                    st_fail++;
                    if (lane == 0)
                        st_rcyc += clock64() - r_t0;
                    int stop = 0;
                    if (lane == 0) {
                        bool done = kServe ? (vld32(&p.ctl->stop) != 0u) : (vld32(&p.ctl->graphs_left) == 0u);
                        // kAcyc: settled by reductions, so the graph is done
                        // when a thief finds nothing pending
                        if (kAcyc && !done && (u32)vld64(&p.descs[p.single_gid].pe) == 0u) {
                            done = true;
                            atomicExch(&p.ctl->graphs_left, 0u);
                        }
                        if (done || vldi(&p.ctl->abort_code) != 0) {
                            stop = 1;
                        } else if (globaltimer() > deadline) {
                            atomicCAS(&p.ctl->abort_code, 0, TG_ERR_TIMEOUT);
                            stop = 1;
                        } else if (p.cancel && (idle & 15u) == 0u && *p.cancel != 0u) {
                            atomicCAS(&p.ctl->abort_code, 0, TG_ERR_CANCELLED);
                            stop = 1;
                        }
                        if (w.err) {
                            atomicCAS(&p.ctl->abort_code, 0, TG_ERR_INTERNAL);
                            stop = 1;
                        }
                        if (stop)
                            *(volatile int *)&s_stop = 1;
                        else if (atomicExch(&s_hungry, 1) == 0)
                            atomicAdd(&p.ctl->hungry, 1u);
                    }
                    if (adaptive) {
                        // the last thief keeps stealing while a block is active or
                        // a queue holds work; any other failed thief parks its
                        // block until a wake ticket (or the end) arrives -- but
                        // only a block with no busy warp: the thief role is the
                        // only way into the block's own public deque, which its
                        // busy warps may still fill
                        const u32 nwa = (p.nblocks + 31u) >> 5;
                        const int any = __ballot_sync(kFull, (u32)lane < nwa && vld32(&p.ctl->avail[lane]) != 0u) != 0 ||
                                        ring_size(w.inj) != 0u;
                        if (lane == 0) {
                            const bool last = atomicSub(&p.ctl->thieves, 1u) == 1u;
                            const bool idle_block = *(volatile u32 *)&s_busy == 0u;
                            if (!stop && idle_block && !(last && (any || vld32(&p.ctl->actives) != 0u))) {
                                st_park++;
                                u32 nap = 256, naps = 0;
                                for (;;) {
                                    __nanosleep(nap);
                                    nap = min(nap * 2u, 4096u);
                                    ++naps;
                                    if (vld32(&p.ctl->graphs_left) == 0u || vldi(&p.ctl->abort_code) != 0) {
                                        stop = 1;
                                    } else if (globaltimer() > deadline) {
                                        atomicCAS(&p.ctl->abort_code, 0, TG_ERR_TIMEOUT);
                                        stop = 1;
                                    } else if (p.cancel && (naps & 15u) == 0u && *p.cancel != 0u) {
                                        atomicCAS(&p.ctl->abort_code, 0, TG_ERR_CANCELLED);
                                        stop = 1;
                                    }
                                    if (stop) {
                                        *(volatile int *)&s_stop = 1;
                                        break;
                                    }
                                    const u32 tk = vld32(&p.ctl->wake);
                                    if (tk != 0u && atomicCAS(&p.ctl->wake, tk, tk - 1u) == tk)
                                        break;
                                    // a warp of this block that was just starting a
                                    // step may still publish to the block's deque
                                    if ((vld32(w.avail_word) & w.avail_bit) != 0u)
                                        break;
                                }
                                backoff = 256;
                            }
                        }
                    }
                    if (lane == 0) {
                        if (!adaptive)
                            vst32(&p.thief_slots[my_slot * 32u], 0u);
                        __threadfence_block();
                        *(volatile int *)&s_thief = 0;
                    }
                    if (__shfl_sync(kFull, stop, 0))
                        break;
                    idle++;
                    __nanosleep(backoff);
                    backoff = min(backoff * 2u, backoff_max);
                    continue;
                }
                if (lane == 0) {
                    if (adaptive) {
                        // the last thief to become active wakes a parked block
                        // to take over its role
                        if (atomicSub(&p.ctl->thieves, 1u) == 1u)
                            atomicAdd(&p.ctl->wake, 1u);
                    } else {
                        vst32(&p.thief_slots[my_slot * 32u], 0u);
                    }
                    *(volatile int *)&s_thief = 0;
                }
                backoff = 256;
            }
        }
        st_iters++;
        mark(0);
        if (count_busy && !busy_w) {
            busy_w = true;
            if (lane == 0 && atomicAdd(&s_busy, 1u) == 0u && adaptive)
                atomicAdd(&p.ctl->actives, 1u);
        }
        if (lane == 0 && *(volatile int *)&s_hungry != 0 && atomicExch(&s_hungry, 0) == 1)
            atomicSub(&p.ctl->hungry, 1u);
        if (lane == 0)
            w.hungry_v = vld32(w.hungry);   // used when the step publishes

        // ---- read the activations' tasks
        bool act = lane < k && (u32)e != kEmpty32;
        if (act && ((u32)e & kIdMask) >= p.node_cap) {
            w.err = 3;   // never produced by the scheduler: treat as a fault, touch nothing
            act = false;
        }
        u32 u = 0, insum = 0;
        bool strong = false;
        if (act) {
            u = (u32)e & kIdMask;
            strong = ((u32)e & kStrongBit) != 0u;
            insum = (u32)(e >> 32);
            if (task_trace) {
                p.trace[3ull * u] = globaltimer();
                p.trace[3ull * u + 2ull] = ((u64)from << 16) | (u64)blockIdx.x;
            }
        }
        uint4 imm = make_uint4(0, 0, 0, 0);
        uint2 stt = make_uint2(0, 0);
        u32 gid = 0;
        if (act) {
            imm = (kAcyc && pre_now) ? hand_imm : ld_imm<kServe>(reinterpret_cast<const uint4 *>(&p.slots[u]));
            // (an acyclic launch runs each task once: its count and digest are 0)
            stt = acyclic ? make_uint2(0u, 0u) : __ldcg(reinterpret_cast<const uint2 *>(&p.slots[u].cnt));
            gid = single ? p.single_gid : ld_imm<kServe>(&p.chunk_gid[u >> kChunkShift]);
        }
        if (act) {
            // the resident server recycles graph slots, so it re-reads the
            // descriptor of every activation
            if (kServe || gid != c_gid || c_age >= 16u) {
                c_seed = ld_imm<kServe>(&p.descs[gid].seed);
                c_cap = ld_imm<kServe>(&p.descs[gid].exec_cap);
                c_base = ld_imm<kServe>(&p.descs[gid].node_off);
                c_status = vldi(&p.descs[gid].status);
                c_gid = gid;
                c_age = 0;
            } else {
                c_age++;
            }
        }
        // a module task's list starts with the slot id of the graph it composes
        const u32 succ_off = imm.x + ((modules && ((imm.z >> 16) & 0xFFu) >= TG_MODULE) ? 1u : 0u);
        const u32 succ_cnt = imm.y & 0xFFFFu;
        const u32 indeg = imm.y >> 16;
        const u32 rounds = imm.z & 0xFFFFu;
        const u32 kind = kAcyc ? (u32)TG_STATIC : ((imm.z >> 16) & 0xFFu);
        const u32 arg = imm.z >> 24;
        const u32 lid = imm.w;
        const u32 iter = stt.x & ~(kInflight | kAwait);
        // a module task whose composed graph finished: release its successors
        const bool cont = modules && act && kind >= TG_MODULE && (stt.x & kAwait) != 0u;
        const bool enter = modules && act && kind >= TG_MODULE && !cont;
        // a detached subflow releases its successors at its first step
        const bool detached = enter && kind == TG_SUBFLOW && (arg & 1u) != 0u;

        // Successor ids of static tasks are fetched before the payload runs,
        // so their latency hides under it.  If no lane has more than
        // kPerLaneMax successors each lane releases its own; otherwise the
        // edges are flattened over the warp (edge e belongs to the lane
        // whose exclusive prefix covers it) to spread a wide fan-out.
        const u32 c = (act && (kind == TG_STATIC || cont || detached)) ? succ_cnt : 0u;
        const u32 maxc = __reduce_max_sync(kFull, c);
        const bool per_lane = maxc <= kPerLaneMax;
        if (traced) {
            asm volatile("" ::"r"(maxc), "r"(iter), "r"(lid), "r"(c_seed));
            mark(1);
        }
        // The loads leave raw successor words in s_; decode() turns them
        // into node-pool ids later, so that the first round's loads stay in
        // flight while the payload runs.
        u32 s_[kRelUnroll], ow_[kRelUnroll];
        bool v_[kRelUnroll];
        u32 total = 0, excl = 0;
        auto fetch_lane = [&](u32 j0) {
#pragma unroll
            for (int j = 0; j < kRelUnroll; ++j) {
                v_[j] = j0 + (u32)j < c;
                ow_[j] = (u32)lane;
                s_[j] = ld_early<kServe>(&p.edges[succ_off + j0 + (u32)j], v_[j]);
            }
        };
        // (the base of the owner's graph: an idle lane may own no graph)
        auto decode = [&]() {
#pragma unroll
            for (int j = 0; j < kRelUnroll; ++j) {
                const u32 base_o = __shfl_sync(kFull, c_base, (int)ow_[j]);
                s_[j] = v_[j] ? (base_o + (s_[j] & ~kSoleBit)) | (s_[j] & kSoleBit) : 0u;
            }
        };
        auto fetch_flat = [&](u32 base) {
#pragma unroll
            for (int j = 0; j < kRelUnroll; ++j) {
                const u32 ei = base + (u32)j * 32u + (u32)lane;
                v_[j] = ei < total;
                const u32 eq = v_[j] ? ei : total - 1u;
                int o = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    u32 ex = __shfl_sync(kFull, excl, o + step);
                    if (ex <= eq)
                        o += step;
                }
                const u32 off_o = __shfl_sync(kFull, succ_off, o);
                const u32 ex_o = __shfl_sync(kFull, excl, o);
                ow_[j] = (u32)o;
                s_[j] = ld_early<kServe>(&p.edges[off_o + (eq - ex_o)], v_[j]);
            }
        };
        if (per_lane) {
            if (maxc)
                fetch_lane(0u);
        } else {
            u32 incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                u32 y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o)
                    incl += y;
            }
            total = __shfl_sync(kFull, incl, 31);
            excl = incl - c;
            fetch_flat(0u);
        }

        // A condition's choice depends on its id and count, not on its
        // output: its successor is fetched before the payload too.
        int c_r = -1;
        u32 c_raw = 0;
        if (!kAcyc && act && c_status == 0 && kind >= TG_COND_BRANCH && kind <= TG_COND_CONST) {
            c_r = cond_index(kind, arg, c_seed, lid, iter, succ_cnt);
            if (c_r >= 0 && (u32)c_r < succ_cnt)
                c_raw = ld_early<kServe>(&p.edges[succ_off + (u32)c_r], true);
            else
                c_r = -1;
        }

        // a strong activation consumed its join word: re-arm it for the next
        // round (composes with releases of that round that arrive early); a
        // task of an acyclic launch has no next round
        if (act && strong && !acyclic)
            atomicAdd(&p.slots[u].W, (u64)indeg - ((u64)insum << 32));

        // ---- payload
        const u32 x = cont ? __ldcg(&p.outv[u]) +
                                 (kind == TG_SUBFLOW ? vld32(&p.descs[ld_imm<kServe>(&p.edges[imm.x])].acc) : 0u)
                           : (act ? task_payload(lid, iter, insum, rounds) : 0u);
        const u32 dg = cont ? stt.y : mix32(stt.y ^ x);
        // a static sink of a subflow copy adds its output to the copy's join value
        const bool sink_acc = modules && act && c_status == 0 && kind == TG_STATIC && succ_cnt == 0u;
        if (sink_acc)
            atomicAdd(&p.descs[gid].acc, x);
        // the previous iteration's pending-count update has arrived meanwhile
        resume(settle_finish<kServe, kExt>(p, pend, pend_old, pend_delta, pend_g, pend_cap), st_spill);
        if (traced) {
            asm volatile("" ::"r"(dg));
            mark(2);
        }

        const bool run = act && c_status == 0;
        const u32 U = run ? ((kind == TG_STATIC || cont) ? succ_cnt : (detached ? succ_cnt + 1u : 1u)) : 0u;
        // acyclic launches of one graph reserve pending counts only for the
        // activations that leave the warp, as they leave it
        u64 *const pe_lazy = kAcyc ? &p.descs[p.single_gid].pe : nullptr;
        // reserve the pending count of every activation this warp may push
        // before any of them becomes visible (a fence precedes publication)
        if (single) {
            if (!kAcyc) {
                const u32 sumU = __reduce_add_sync(kFull, U);
                if (lane == 0 && sumU)
                    atomicAdd(&p.descs[p.single_gid].pe, (u64)sumU);
            }
        } else {
            // lanes grouped by graph (lanes that run nothing form one more
            // group); each group's lowest lane adds the group's sum
            const u32 m = __match_any_sync(kFull, run ? gid : kEmpty32);
            const u32 sumU = __reduce_add_sync(m, U);
            if (run && sumU && lane == __ffs(m) - 1)
                atomicAdd(&p.descs[gid].pe, (u64)sumU);
        }
        if (run && !cont)
            st_tasks++;
        // A task that can run again stores its output before its releases,
        // which are what make a later execution of it (on another SM)
        // possible.  Issued after them, the store was seen to land after the
        // next execution's under heavy stealing, leaving a stale final
        // output.  (Without in-flight flags the fence below orders it; with
        // them, the flag release comes a full round of release and
        // push-check atomics after it.)
        if (!acyclic && run && !cont)
            __stcs(&p.outv[u], x);
        if (!race_check && !acyclic) {
            // without in-flight flags the state must be visible before any
            // release makes a later activation of this task possible
            if (run)
                __stcg(reinterpret_cast<uint2 *>(&p.slots[u].cnt),
                       make_uint2(cont ? iter : ((iter + 1u) | (enter ? kAwait : 0u)), dg));
            fence_acq_rel_gpu();
        }
        if (!per_lane) {
            my_push[lane] = 0;
            my_keep[lane] = 0;
        }
        __syncwarp();

        // New activations are staged in shared memory.  Each target's
        // in-flight flag is set (and checked) first; this task's own flag is
        // released -- together with its new count and digest -- only after
        // all of its checks returned, and only then are the activations
        // published.  A task that pushes itself hands its flag on.
        u32 ns = 0;              // staged entries (warp-uniform)
        u32 kept = 0;            // of them, kept by the warp for its next step
        u32 racy = kEmpty32;     // graph whose activation found a target in flight
        u32 mp = 0;              // activations this lane's task pushed (own-lane part)
        bool keep_self = false;  // this lane's task pushed itself

        // ---- condition tasks: jump to successors[r]
        bool c_has = false;
        u32 c_t = 0, c_fl = 0;
        if (run && c_r >= 0) {
            c_t = c_base + (c_raw & ~kSoleBit);
            c_has = true;
            mp++;
            if (race_check) {
                if (c_t == u)
                    keep_self = true;
                else
                    c_fl = atomicOr(&p.slots[c_t].cnt, kInflight);
            }
        }

        // ---- static tasks: release every successor
        if (per_lane) {
            for (u32 j0 = 0; j0 < maxc; j0 += kRelUnroll) {
                if (j0)
                    fetch_lane(j0);
                decode();
                u64 old_[kRelUnroll];
                u32 fl_[kRelUnroll];
                bool has_[kRelUnroll];
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j) {
                    v_[j] = v_[j] && run;
                    // a target with no other strong in-edge is ready at once,
                    // with this task's output as its input sum
                    old_[j] = (v_[j] && (s_[j] & kSoleBit) == 0u)
                                  ? atomicAdd(&p.slots[s_[j]].W, ((u64)x << 32) - 1ull) : 0ull;
                }
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j) {
                    const bool sole = (s_[j] & kSoleBit) != 0u;
                    const u32 t = s_[j] & ~kSoleBit;
                    fl_[j] = 0u;
                    has_[j] = v_[j] && (sole || (u32)old_[j] == 1u);
                    if (has_[j]) {
                        mp++;
                        if (race_check) {
                            if (t == u)
                                keep_self = true;
                            else
                                fl_[j] = atomicOr(&p.slots[t].cnt, kInflight);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j) {
                    const u32 t = s_[j] & ~kSoleBit;
                    const u64 ent = (s_[j] & kSoleBit) ? (((u64)x << 32) | (u64)t)
                                                       : (((u64)((u32)(old_[j] >> 32) + x) << 32) | kStrongBit | (u64)t);
                    stage(w, my_stage, ns, has_[j], ent, lane, st_spill, pe_lazy);
                    if (fl_[j] & kInflight)
                        racy = gid;
                }
            }
        } else {
            // software-pipelined rounds: while a round's join-word atomics are
            // in flight the previous round's race checks are examined, and the
            // next round's successor ids are fetched before this round stages
            u32 pfl_[kRelUnroll], pgo_[kRelUnroll];
#pragma unroll
            for (int j = 0; j < kRelUnroll; ++j) {
                pfl_[j] = 0u;
                pgo_[j] = 0u;
            }
            for (u32 base = 0; base < total; base += 32u * kRelUnroll) {
                u32 xo_[kRelUnroll], go_[kRelUnroll], fl_[kRelUnroll];
                u64 old_[kRelUnroll], ent_[kRelUnroll];
                bool has_[kRelUnroll];
                decode();
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j) {
                    xo_[j] = __shfl_sync(kFull, x, (int)ow_[j]);
                    go_[j] = __shfl_sync(kFull, gid, (int)ow_[j]);
                    const int run_o = __shfl_sync(kFull, (int)run, (int)ow_[j]);   // every lane shuffles
                    v_[j] = v_[j] && run_o != 0;
                }
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j)
                    old_[j] = (v_[j] && (s_[j] & kSoleBit) == 0u)
                                  ? atomicAdd(&p.slots[s_[j]].W, ((u64)xo_[j] << 32) - 1ull) : 0ull;
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j)
                    if (pfl_[j] & kInflight)
                        racy = pgo_[j];
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j) {
                    const u32 uo = __shfl_sync(kFull, u, (int)ow_[j]);
                    const bool sole = (s_[j] & kSoleBit) != 0u;
                    const u32 t = s_[j] & ~kSoleBit;
                    fl_[j] = 0u;
                    has_[j] = v_[j] && (sole || (u32)old_[j] == 1u);
                    if (has_[j]) {
                        atomicAdd(&my_push[ow_[j]], 1u);
                        if (race_check) {
                            if (t == uo)
                                my_keep[ow_[j]] = 1u;
                            else
                                fl_[j] = atomicOr(&p.slots[t].cnt, kInflight);
                        }
                    }
                    ent_[j] = sole ? (((u64)xo_[j] << 32) | (u64)t)
                                   : (((u64)((u32)(old_[j] >> 32) + xo_[j]) << 32) | kStrongBit | (u64)t);
                    pfl_[j] = fl_[j];
                    pgo_[j] = go_[j];
                }
                if (base + 32u * kRelUnroll < total)
                    fetch_flat(base + 32u * kRelUnroll);
#pragma unroll
                for (int j = 0; j < kRelUnroll; ++j)
                    stage(w, my_stage, ns, has_[j], ent_[j], lane, st_spill, pe_lazy);
            }
#pragma unroll
            for (int j = 0; j < kRelUnroll; ++j)
                if (pfl_[j] & kInflight)
                    racy = pgo_[j];
        }
        stage(w, my_stage, ns, c_has, ((u64)x << 32) | (u64)c_t, lane, st_spill);
        if (c_fl & kInflight)
            racy = gid;
        if (traced) {
            asm volatile("" ::"r"(racy), "r"(ns), "r"(mp));
            mark(3);
        }
        __syncwarp();
        if (!per_lane) {
            mp += my_push[lane];
            keep_self = keep_self || my_keep[lane] != 0u;
        }

        // ---- a race poisons the graph in which it was found
        if (racy != kEmpty32)
            atomicCAS(&p.descs[racy].status, 0, TG_ERR_RACE);

        if (enter && run)
            mp++;   // a module task's continuation, or a detached copy's token of this graph

        // ---- release own in-flight flags (with the new count and digest).
        // The fence orders them, and the pending-count reservation, before
        // the publication of new work; a step that publishes nothing (it
        // keeps its output in hand) leaves it to the next step that does.
        // The flag release must reach L2 before any later activation of the
        // task can test it there (an atomic, which a block-scope fence does
        // not order against a plain store): GPU scope.  An acyclic launch
        // has no flags and its tasks run once, so there the only ordering
        // is the reservation's, for the block's own ring: block scope
        // (activations that leave the block are fenced GPU-wide where they
        // are pushed, in emit).  The server always fences GPU-wide: the host
        // reads its completion records while it runs.  A module task keeps
        // its flag (and marks itself waiting) until its continuation has run.
        const bool any_enter = modules && __any_sync(kFull, (enter && run) || sink_acc);
        if (race_check || acyclic) {
            if (run)
                __stcg(reinterpret_cast<uint2 *>(&p.slots[u].cnt),
                       make_uint2((cont ? iter : iter + 1u) | (keep_self ? kInflight : 0u) |
                                      ((enter && !detached) ? (kInflight | kAwait) : 0u),
                                  dg));
            if (kServe || any_enter || (ns > kHandMax && !acyclic))
                fence_acq_rel_gpu();
            else if (ns > kHandMax && !kAcyc)
                fence_acq_rel_cta();
        } else if (any_enter) {
            fence_acq_rel_gpu();
        }
        if (acyclic && run)
            __stcs(&p.outv[u], x);
        if (any_enter) {
            // ---- a module task enters its composed graph: takes it (its
            // pending count must be idle, else two module tasks use it at
            // once: a race), names itself as the task to resume, and -- after
            // a fence -- activates the graph's sources with its output.  A
            // refused entry resumes at once.
            bool entered = false;
            u32 m_base = 0, m_src = 0, m_nsrc = 0, m_n = 0, m_g = 0;
            if (enter && run) {
                m_g = ld_imm<kServe>(&p.edges[imm.x]);
                m_nsrc = ld_imm<kServe>(&p.descs[m_g].n_src);
                m_src = ld_imm<kServe>(&p.descs[m_g].src_off);
                m_base = ld_imm<kServe>(&p.descs[m_g].node_off);
                m_n = ld_imm<kServe>(&p.descs[m_g].n);
                const u64 was = atomicAdd(&p.descs[m_g].pe, (u64)m_nsrc);
                if ((u32)was == 0u) {
                    vst32(&p.descs[m_g].ret, u | (detached ? kDetachBit : 0u));
                    if (kind == TG_SUBFLOW) {
                        // a fresh copy: no executions, no status, no join value yet
                        vst64(&p.descs[m_g].pe, (u64)m_nsrc);
                        vst32((u32 *)&p.descs[m_g].status, 0u);
                        vst32(&p.descs[m_g].acc, 0u);
                    }
                    entered = true;
                } else {
                    atomicAdd(&p.descs[m_g].pe, (u64)0 - (u64)m_nsrc);
                    atomicCAS(&p.descs[gid].status, 0, TG_ERR_RACE);
                    if (detached)
                        atomicAdd(&p.descs[gid].pe, ~0ull);   // no copy holds the token
                }
            }
            // a subflow copy's tasks start from their initial state
            {
                u32 rs = __ballot_sync(kFull, entered && kind == TG_SUBFLOW);
                while (rs) {
                    const int l = __ffs(rs) - 1;
                    rs &= rs - 1u;
                    const u32 nb = __shfl_sync(kFull, m_base, l);
                    const u32 nn = __shfl_sync(kFull, m_n, l);
                    for (u32 i = (u32)lane; i < nn; i += 32u) {
                        NodeSlot *sl = &p.slots[nb + i];
                        vst64(&sl->W, (u64)(ld_imm<kServe>(&sl->deg) >> 16));
                        vst64(reinterpret_cast<u64 *>(&sl->cnt), 0ull);
                    }
                }
            }
            fence_acq_rel_gpu();
            emit(w, enter && run && !entered && !detached, (u64)u, lane, st_spill);
            u32 rem = __ballot_sync(kFull, entered);
            while (rem) {
                const int l = __ffs(rem) - 1;
                rem &= rem - 1u;
                const u32 nb = __shfl_sync(kFull, m_base, l);
                const u32 so = __shfl_sync(kFull, m_src, l);
                const u32 nn = __shfl_sync(kFull, m_nsrc, l);
                const u32 xv = __shfl_sync(kFull, x, l);
                for (u32 i = 0; i < nn; i += 32u) {
                    const bool h = i + (u32)lane < nn;
                    const u64 ent = h ? (((u64)xv << 32) | (u64)(nb + __ldcg(&p.edges[so + i + (u32)lane]))) : 0ull;
                    emit(w, h, ent, lane, st_spill);
                }
            }
        }
        if (task_trace && act)
            p.trace[3ull * u + 1ull] = globaltimer();
        // ---- a warp whose step produced at most kHandMax activations runs
        // them itself next (a chain never leaves the warp); wider output is
        // published to the block's ring / public deque, where it merges with
        // the siblings' work and spreads.  With hand_batch a whole step's
        // output up to batch_max stays with the warp while the block's ring
        // is empty (no sibling waits for work there): on a wavefront it then
        // skips the publication and the pickup of every hop.
        {
            u32 keep = ns <= kHandMax ? ns : 0u;
            kept = 0u;
            if (p.hand_batch && keep == 0u && ns <= (u32)bmax) {
                u32 lsz = 0;
                if (lane == 0)
                    lsz = ring_size<true>(w.local);
                if (__shfl_sync(kFull, lsz, 0) == 0u)
                    keep = ns;
            }
            __syncwarp();
            hand = (u32)lane < keep ? my_stage[lane] : kEmpty;
            nh = (int)keep;
            // kAcyc: the kept tasks' records are loaded now, their latency
            // hidden behind the rest of this step (records are immutable
            // while the graph runs)
            hand_pre = false;
            if (kAcyc && keep) {
                if ((u32)lane < keep)
                    hand_imm = ld_imm<kServe>(reinterpret_cast<const uint4 *>(&p.slots[(u32)hand & kIdMask]));
                hand_pre = true;
            }
            kept = keep;
            if (ns > keep) {
                if (kAcyc) {
                    if (lane == 0)
                        atomicAdd(pe_lazy, (u64)(ns - keep));
                    fence_acq_rel_cta();
                }
                publish<kIdle>(w, my_stage + keep, ns - keep, lane, st_spill, pe_lazy);
            }
            __syncwarp();
        }

        // ---- settle the pending counts: + pushed - reserved - executed.
        // The atomic's result is examined next iteration (settle_finish).
        {
            const u32 P = act ? mp : 0u;
            if (single) {
                const u32 E = (u32)__popc(__ballot_sync(kFull, act));
                const u32 sumP = __reduce_add_sync(kFull, P);
                const u32 sumU = __reduce_add_sync(kFull, U);
                if (lane == 0 && E) {
                    // (kAcyc: what left the warp was reserved as it left)
                    const long long d = kAcyc ? (long long)kept - (long long)E
                                              : (long long)sumP - (long long)sumU - (long long)E;
                    pend_delta = ((u64)E << 32) + (u64)d;   // (no continuations without modules)
                    if (kAcyc) {
                        // every task runs at most once, so the cap needs no
                        // check on the way: a reduction (its returned value
                        // would hold the warp up), and idle thieves notice
                        // the pending count reach zero
                        atomicAdd(&p.descs[p.single_gid].pe, pend_delta);
                    } else {
                        pend_old = atomicAdd(&p.descs[p.single_gid].pe, pend_delta);
                        pend_g = p.single_gid;
                        pend_cap = single_cap;
                        pend = true;
                    }
                }
            } else {
                // one pending-count update per graph of the step, by the
                // lowest lane of the graph's group (as for the reservation)
                const u32 m = __match_any_sync(kFull, act ? gid : kEmpty32);
                // a continuation consumes its pending count but is no execution
                const u32 mx = __ballot_sync(kFull, act && !cont) & m;
                const u32 sumP = __reduce_add_sync(m, P);
                const u32 sumU = __reduce_add_sync(m, U);
                if (act && lane == __ffs(m) - 1) {
                    const u32 E = (u32)__popc(m);
                    const long long d = (long long)sumP - (long long)sumU - (long long)E;
                    pend_delta = ((u64)__popc(mx) << 32) + (u64)d;
                    pend_old = atomicAdd(&p.descs[gid].pe, pend_delta);
                    pend_g = gid;
                    pend_cap = c_cap;
                    pend = true;
                }
            }
        }
        mark(4);
        // a bounded wait that gave up (any lane): the whole warp stops
        if (__any_sync(kFull, w.err != 0)) {
            if (lane == 0)
                atomicCAS(&p.ctl->abort_code, 0, TG_ERR_INTERNAL);
            break;
        }
        // a busy warp also honours the time limit and aborts
        if ((st_iters & 63u) == 0u) {
            int stop = 0;
            if (lane == 0) {
                if (vldi(&p.ctl->abort_code) != 0)
                    stop = 1;
                else if (globaltimer() > deadline) {
                    atomicCAS(&p.ctl->abort_code, 0, TG_ERR_TIMEOUT);
                    stop = 1;
                }
            }
            if (__shfl_sync(kFull, stop, 0))
                break;
        }
    }

    (void)settle_finish<kServe, kExt>(p, pend, pend_old, pend_delta, pend_g, pend_cap);
    if (lane == 0) {
        atomicAdd(&s_stats[ST_POP_LOCAL], st_local);
        atomicAdd(&s_stats[ST_POP_OWN], st_own);
        atomicAdd(&s_stats[ST_STEAL_TRY], st_try);
        atomicAdd(&s_stats[ST_STEAL_HIT], st_hit);
        atomicAdd(&s_stats[ST_INJECT], st_inj);
        atomicAdd(&s_stats[ST_SPILL], st_spill);
        atomicAdd(&s_stats[ST_IDLE], st_idle);
        atomicAdd(&s_stats[ST_ITERS], st_iters);
        atomicAdd(&s_stats[ST_HAND], st_hand);
        atomicAdd(&s_stats[ST_PARK], st_park);
        atomicAdd(&s_stats[ST_FAILED_ROUND], st_fail);
        atomicAdd(&s_stats[ST_ROUND_CYCLES], st_rcyc);
    }
    // tasks are counted per lane
    atomicAdd(&s_stats[ST_TASKS], st_tasks);
    __syncthreads();
    if (threadIdx.x == 0)
        s_stats[ST_PEAK_THIEVES] = s_peak;
    __syncthreads();
    if (threadIdx.x < ST_COUNT)
        p.stats[(size_t)blockIdx.x * ST_COUNT + threadIdx.x] = s_stats[threadIdx.x];
}

// One-shot launches (single graphs, batches): at most 512 threads (16 worker
// warps), so that 128 registers per thread fill the SM.  kOne: one graph;
// kAcyc: one graph without condition tasks (every task static, run once);
// kTrace: records per-task trace words (TG_OPT_TRACE_TASKS), a copy of the
// lean variant so that untraced launches carry none of it; kIdle: keep_idle
// (one graph with condition tasks).
template <bool kExt, bool kOne, bool kAcyc = false, bool kTrace = false, bool kIdle = false>
__global__ void __launch_bounds__(512, 1) sched_kernel(KParams p)
{
    sched_body<false, kExt, kOne, kAcyc, kTrace, kIdle>(p);
}

// every one-shot variant: they share the block shape a geometry allows
using SchedFn = void (*)(KParams);
const SchedFn kOneShotVariants[] = {
    sched_kernel<true, false>,        sched_kernel<false, true>,        sched_kernel<false, true, true>,
    sched_kernel<false, false>,       sched_kernel<false, true, false, true>, sched_kernel<false, true, true, true>,
    sched_kernel<false, false, false, true>, sched_kernel<false, true, false, false, true>,
};

// The resident server (its blocks are at most half an SM).
__global__ void serve_kernel(KParams p)
{
    sched_body<true, false, false>(p);
}

// ---------------------------------------------------------------------------
// re-arm: state of every graph of the launch, queues, sources (Algorithm 8)
// grid = (ceil(max_n / 1024), n_graphs)
// ---------------------------------------------------------------------------
__global__ void rearm_kernel(KParams p)
{
    const u32 gi = blockIdx.y;
    const u32 gid = p.lt ? p.lt[gi].gid : p.single_gid;
    const u32 inj_base = p.lt ? p.lt[gi].inj_base : 0u;
    GDesc &D = p.descs[gid];
    const u32 n = D.n;
    const u32 off = D.node_off;
    const u32 first = blockIdx.x * 1024u;
    for (u32 i = first + threadIdx.x; i < n && i < first + 1024u; i += blockDim.x) {
        const u32 u = off + i;
        const u32 deg = p.slots[u].deg;
        p.slots[u].W = (u64)(deg >> 16);
        *reinterpret_cast<uint2 *>(&p.slots[u].cnt) = make_uint2(0u, 0u);
        p.outv[u] = 0u;
        if (p.trace) {
            p.trace[3ull * u] = 0ull;
            p.trace[3ull * u + 1ull] = 0ull;
            p.trace[3ull * u + 2ull] = 0ull;
        }
    }
    // the successor lists of this block's tasks are pulled into L2 ahead of
    // the scheduler, which reads each once, on its critical path
    if (first < n) {
        const u32 last = min(n, first + 1024u);
        const u32 lo = p.slots[off + first].succ_off;
        const u32 hi = last < n ? p.slots[off + last].succ_off : D.src_off;
        for (u32 w = (lo & ~31u) + threadIdx.x * 32u; w < hi; w += blockDim.x * 32u)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p.edges + w));
    }
    if (blockIdx.x == 0) {
        for (u32 s = threadIdx.x; s < D.n_src; s += blockDim.x)
            p.inj[(inj_base + s) & p.inj_mask] = (u64)(D.node_off + p.edges[D.src_off + s]);
        if (threadIdx.x == 0) {
            D.pe = (u64)D.n_src;
            D.status = 0;
            D.ret = kEmpty32;
        }
    }
    if (gi == 0 && blockIdx.x == 0) {
        for (u32 b = threadIdx.x; b < p.nblocks; b += blockDim.x) {
            p.dqc[b].head = 0u;
            p.dqc[b].tail = 0u;
        }
        for (u32 i = threadIdx.x; i < p.nblocks * (u32)ST_COUNT; i += blockDim.x)
            p.stats[i] = 0ull;
        for (u32 i = threadIdx.x; i < p.max_thieves; i += blockDim.x)
            p.thief_slots[i * 32u] = 0u;
        for (u32 i = threadIdx.x; i < 32u; i += blockDim.x)
            p.ctl->avail[i] = 0u;
        if (threadIdx.x == 0) {
            p.ctl->graphs_left = p.n_graphs;
            p.ctl->abort_code = 0;
            p.ctl->hungry = 0u;
            p.ctl->actives = 0u;
            p.ctl->thieves = 0u;
            p.ctl->wake = 0u;
            p.ctl->inj.head = 0u;
            p.ctl->inj.tail = p.total_sources;
            if (p.cancel)
                *p.cancel = 0u;
        }
    }
}

// An instance's records from its template's (immutable half read through
// L2: the template may be running, which changes only the other half).
__global__ void instance_rearm_kernel(NodeSlot *slots, u64 src_off, u64 dst_off, u32 n)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 imm = __ldcg(reinterpret_cast<const uint4 *>(&slots[src_off + i]));
        uint4 *d = reinterpret_cast<uint4 *>(&slots[dst_off + i]);
        d[0] = imm;
        d[1] = make_uint4(imm.y >> 16, 0u, 0u, 0u);   // W = {insum 0 | strong in-degree}, cnt, dig
    }
}

// A graph composed by a module task of the launch: its state starts from
// scratch, idle (nothing pending, no module task to resume), sources not
// activated -- its module task does that.
__global__ void module_rearm_kernel(KParams p, u32 gid, u32 n)
{
    GDesc &D = p.descs[gid];
    const u32 off = D.node_off;
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const u32 u = off + i;
        p.slots[u].W = (u64)(p.slots[u].deg >> 16);
        *reinterpret_cast<uint2 *>(&p.slots[u].cnt) = make_uint2(0u, 0u);
        p.outv[u] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        D.pe = 0ull;
        D.status = 0;
        D.ret = kEmpty32;
        D.acc = 0u;
    }
}

// After the scheduler: unfinished graphs take the launch's abort code; every
// status is mirrored to host-mapped memory.  An aborted launch (time limit,
// cancel, internal error) may leave activations in its queues; they are
// emptied here, so that the next launch on the stream starts from empty
// slots whether or not the host has seen this launch's status yet.
__global__ void finalize_kernel(KParams p)
{
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 nthreads = gridDim.x * blockDim.x;
    for (u32 gi = tid; gi < p.n_graphs; gi += nthreads) {
        const u32 gid = p.lt ? p.lt[gi].gid : p.single_gid;
        GDesc &D = p.descs[gid];
        i32 st = D.status;
        if (st == 0 && (u32)D.pe != 0u) {
            i32 ab = p.ctl->abort_code;
            st = ab != 0 ? ab : TG_ERR_INTERNAL;
            D.status = st;
        }
        // (the lean kernel for a graph without condition tasks counts
        // executions without checking them against the cap as it goes)
        if (st == 0 && (u32)(D.pe >> 32) > D.exec_cap) {
            st = TG_ERR_EXEC_LIMIT;
            D.status = st;
        }
        if (p.status_out)
            p.status_out[gid] = st;
    }
    if (p.ctl->abort_code != 0) {
        for (size_t i = tid; i <= (size_t)p.inj_mask; i += nthreads)
            p.inj[i] = kEmpty;
        const size_t dq_slots = (size_t)p.nblocks * p.dq_stride;
        for (size_t i = tid; i < dq_slots; i += nthreads)
            p.dq[i] = kEmpty;
    }
}

__global__ void clear_kernel(u64 *slots, size_t count)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        slots[i] = kEmpty;
}

// ---------------------------------------------------------------------------
// roofline kernels
// ---------------------------------------------------------------------------
// The payload alone on ids 0..count-1 (iter 0, insum 0): the integer-ALU
// ceiling of the scheduler's execute step.  Four independent chains per
// thread give the issue slots enough independent work.
__global__ void bench_payload_kernel(u64 count, u32 rounds, u32 *checksum)
{
    const u64 stride = (u64)gridDim.x * blockDim.x;
    u32 acc = 0;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < count; i += 4 * stride) {
        u32 a = task_payload((u32)i, 0u, 0u, rounds);
        u32 b = i + stride < count ? task_payload((u32)(i + stride), 0u, 0u, rounds) : 0u;
        u32 c = i + 2 * stride < count ? task_payload((u32)(i + 2 * stride), 0u, 0u, rounds) : 0u;
        u32 d = i + 3 * stride < count ? task_payload((u32)(i + 3 * stride), 0u, 0u, rounds) : 0u;
        acc ^= a ^ b ^ c ^ d;
    }
    for (int o = 16; o; o >>= 1)
        acc ^= __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0)
        atomicXor(checksum, acc);
}

// The payload alone over a given multiset of executions: thread i runs task
// i's cnt[i] payloads (iterations 0..cnt[i]-1) of rounds[i] rounds on id
// ids[i].  The arrays' order decides which executions share a warp.
__global__ void bench_payload_tasks_kernel(u32 n, const u32 *ids, const u32 *rounds, const u32 *cnt, u32 *checksum)
{
    u32 acc = 0;
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const u32 id = ids[i], R = rounds[i], c = cnt[i];
        for (u32 it = 0; it < c; ++it)
            acc ^= task_payload(id, it, 0u, R);
    }
    for (int o = 16; o; o >>= 1)
        acc ^= __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0)
        atomicXor(checksum, acc);
}

// The compute along a path of `hops` dependent tasks, with nothing else.
__global__ void bench_chain_kernel(u32 hops, u32 rounds, u32 *last)
{
    u32 x = 0;
    for (u32 h = 0; h < hops; ++h)
        x = task_payload(h, 0u, x, rounds);
    *last = x;
}

// One task of a captured DAG (Algorithm 1): its predecessors ran before it
// on this or another stream, and each added its output to the task's join
// word; the task runs once and passes its output on the same way.
__global__ void capture_task_kernel(NodeSlot *slots, u32 *outv, const u32 *edges, u32 u, u32 node_off)
{
    const NodeSlot &s = slots[u];
    const u32 succ_off = s.succ_off;
    const u32 succ_cnt = s.deg & 0xFFFFu;
    const u32 insum = (u32)(vld64(&slots[u].W) >> 32);
    const u32 x = task_payload(s.lid, 0u, insum, s.prm & 0xFFFFu);
    for (u32 j = threadIdx.x; j < succ_cnt; j += blockDim.x)
        atomicAdd(&slots[node_off + (edges[succ_off + j] & ~kSoleBit)].W, (u64)x << 32);
    if (threadIdx.x == 0) {
        outv[u] = x;
        *reinterpret_cast<uint2 *>(&slots[u].cnt) = make_uint2(1u, mix32(x));
    }
}

// `count` returning 64-bit atomicAdd at pseudo-random words of a footprint.
__global__ void bench_atomics_kernel(u64 *words, u64 footprint, u64 count, u64 *sink)
{
    const u64 stride = (u64)gridDim.x * blockDim.x;
    u64 acc = 0;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < count; i += stride) {
        u32 h = mix32((u32)i ^ mix32((u32)(i >> 32) + 0x51ED27u));
        u64 a = ((u64)h * footprint) >> 32;
        acc += atomicAdd(&words[a], 0x100000001ull);
    }
    if (acc == 0x123456789ull)
        *sink = acc;
}

}  // namespace

size_t sched_dyn_smem(u32 smem_entries, u32 warps)
{
    return ((size_t)smem_entries + (size_t)warps * kStage) * sizeof(u64);
}

cudaError_t sched_occupancy(int threads, size_t dyn_smem, int *blocks_per_sm, bool serve)
{
    // The dynamic shared-memory limit of a kernel is a per-device attribute:
    // it only ever rises, so that a smaller block shape checked here (a
    // server, another context) never invalidates a larger one in use.
    static std::mutex mu;
    static size_t raised[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dyn_smem > raised[dev]) {
            for (SchedFn f : kOneShotVariants) {
                e = cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
                if (e != cudaSuccess)
                    return e;
            }
            e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
            if (e != cudaSuccess)
                return e;
            raised[dev] = dyn_smem;
        }
    }
    if (serve)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, serve_kernel, threads, dyn_smem);
    // every variant must fit the same block shape
    int fewest = 1 << 30;
    for (SchedFn f : kOneShotVariants) {
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, (const void *)f, threads, dyn_smem);
        if (e != cudaSuccess)
            return e;
        fewest = std::min(fewest, b);
    }
    *blocks_per_sm = fewest;
    return cudaSuccess;
}

cudaError_t launch_rearm(const KParams &p, cudaStream_t st)
{
    dim3 grid((p.max_n + 1023u) / 1024u, p.n_graphs);
    if (grid.x == 0)
        grid.x = 1;
    rearm_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_module_rearm(const KParams &p, u32 gid, u32 n, cudaStream_t st)
{
    const u32 blocks = n ? min((n + 255u) / 256u, 4096u) : 1u;
    module_rearm_kernel<<<blocks, 256, 0, st>>>(p, gid, n);
    return cudaGetLastError();
}

cudaError_t launch_sched(const KParams &p, int blocks, int threads, cudaStream_t st, bool serve)
{
    const size_t smem = sched_dyn_smem(p.smem_mask + 1u, (u32)threads / 32u);
    if (serve)
        serve_kernel<<<blocks, threads, smem, st>>>(p);
    else
        if (p.has_modules || p.thief_mode == 1u || (p.flags & TG_OPT_TRACE) != 0u)
            sched_kernel<true, false><<<blocks, threads, smem, st>>>(p);
        else if (p.trace != nullptr && p.lt == nullptr && (p.flags & kFlagAcyclic) != 0u)
            sched_kernel<false, true, true, true><<<blocks, threads, smem, st>>>(p);
        else if (p.trace != nullptr && p.lt == nullptr)
            sched_kernel<false, true, false, true><<<blocks, threads, smem, st>>>(p);
        else if (p.trace != nullptr)
            sched_kernel<false, false, false, true><<<blocks, threads, smem, st>>>(p);
        else if (p.lt == nullptr && (p.flags & kFlagAcyclic) != 0u)
            sched_kernel<false, true, true><<<blocks, threads, smem, st>>>(p);
        else if (p.lt == nullptr && p.keep_idle != 0u)
            sched_kernel<false, true, false, false, true><<<blocks, threads, smem, st>>>(p);
        else if (p.lt == nullptr)
            sched_kernel<false, true><<<blocks, threads, smem, st>>>(p);
        else
            sched_kernel<false, false><<<blocks, threads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const KParams &p, cudaStream_t st)
{
    u32 blocks = (p.n_graphs + 255u) / 256u;
    finalize_kernel<<<blocks ? blocks : 1u, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_clear(u64 *slots, size_t count, cudaStream_t st)
{
    if (count == 0)
        return cudaSuccess;
    size_t blocks = (count + 255) / 256;
    if (blocks > 65535)
        blocks = 65535;
    clear_kernel<<<(unsigned)blocks, 256, 0, st>>>(slots, count);
    return cudaGetLastError();
}

cudaError_t launch_bench_payload(u64 count, u32 rounds, u32 *checksum, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bench_payload_kernel<<<sms * 8, 256, 0, st>>>(count, rounds, checksum);
    return cudaGetLastError();
}

cudaError_t launch_bench_payload_tasks(u32 n, const u32 *ids, const u32 *rounds, const u32 *cnt, u32 *checksum,
                                       cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    bench_payload_tasks_kernel<<<(n + 255u) / 256u, 256, 0, st>>>(n, ids, rounds, cnt, checksum);
    return cudaGetLastError();
}

cudaError_t launch_bench_atomics(u64 *words, u64 footprint, u64 count, u64 *sink, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bench_atomics_kernel<<<sms * 8, 256, 0, st>>>(words, footprint, count, sink);
    return cudaGetLastError();
}

cudaError_t launch_bench_chain(u32 hops, u32 rounds, u32 *last, cudaStream_t st)
{
    bench_chain_kernel<<<1, 1, 0, st>>>(hops, rounds, last);
    return cudaGetLastError();
}

cudaError_t launch_instance_rearm(NodeSlot *slots, u64 src_off, u64 dst_off, u32 n, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    const u32 blocks = min((n + 255u) / 256u, 2048u);
    instance_rearm_kernel<<<blocks, 256, 0, st>>>(slots, src_off, dst_off, n);
    return cudaGetLastError();
}

cudaError_t preload_serving_kernels(cudaStream_t st)
{
    instance_rearm_kernel<<<1, 32, 0, st>>>(nullptr, 0ull, 0ull, 0u);   // n = 0: touches nothing
    return cudaGetLastError();
}

cudaError_t launch_capture_task(NodeSlot *slots, u32 *outv, const u32 *edges, u32 u, u32 node_off, cudaStream_t st)
{
    capture_task_kernel<<<1, 32, 0, st>>>(slots, outv, edges, u, node_off);
    return cudaGetLastError();
}

}  // namespace tg
