// tg_pack.cu -- graph ingest, validation and CSR pack on the device
// (tg_graph_create_dev).
//
// The same checks and the same packed form as the host packer in
// tg_host.cpp (Task Graph Representation; Algorithm 8 reads that form):
//   1. per task: a known kind (static or condition), a loop trip >= 1;
//   2. per edge: both ends < n; out-degree, strong and weak in-degree
//      counted with atomics; explicit edge kinds compared with "the source
//      task is a condition";
//   3. per task: a condition has a successor, degrees <= 65535, and the
//      sources (no strong and no weak in-edge) are flagged;
//   4. the successor lists in insertion order: a stable LSD radix sort of the
//      edges by source task (8 bits a pass), which leaves each task's
//      successors in the order their edges were given -- the order a
//      condition's returned index refers to;
//   5. the 32-byte task records (successor offset = exclusive scan of the
//      out-degrees), the successor ids with the sole-predecessor bit, the
//      source list in task order, the chunk table and the descriptor.
// Every index a kernel writes through was checked (step 2) or computed from
// counts (steps 4-5) before it is used.
#include "../../include/tg.h"
#include "tg_internal.h"

namespace tg {
namespace {

constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr u32 kScanThreads = 1024;
constexpr u32 kScanPer = 8;                              // elements per thread
constexpr u32 kScanChunk = kScanThreads * kScanPer;      // elements per scan block
constexpr u32 kSortWarps = 8;
constexpr u32 kSortRounds = 16;
constexpr u32 kSortTile = kSortWarps * kSortRounds * 32; // 4096 edges per sort block

__device__ __forceinline__ bool pk_cond(u32 kind) { return kind >= TG_COND_BRANCH && kind <= TG_COND_CONST; }

__device__ __forceinline__ u32 grid_stride() { return gridDim.x * blockDim.x; }

// ---- step 1: kinds and loop trips; the conditions are counted
__global__ void pk_nodes_kernel(const u8 *kinds, const u32 *params, u32 n, u32 *flags)
{
    u32 nc = 0;
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += grid_stride()) {
        const u32 k = kinds[v];
        if (k > TG_COND_CONST || (k == TG_COND_LOOP && ((params[v] >> 16) & 0xFFu) == 0u))
            atomicOr(&flags[PK_INVALID], 1u);
        nc += pk_cond(k) ? 1u : 0u;
    }
    nc = __reduce_add_sync(kAll, nc);
    if ((threadIdx.x & 31) == 0 && nc)
        atomicAdd(&flags[PK_NCOND], nc);
}

// ---- step 2: degrees (an edge with an end out of range is only flagged)
__global__ void pk_edges_kernel(const u8 *kinds, const u32 *src, const u32 *dst, const u8 *weak, u32 n, u32 m,
                                u32 *outdeg, u32 *sin, u32 *win, u32 *flags)
{
    for (u32 e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += grid_stride()) {
        const u32 s = src[e], d = dst[e];
        if (s >= n || d >= n) {
            atomicOr(&flags[PK_INVALID], 1u);
            continue;
        }
        const bool c = pk_cond(kinds[s]);
        atomicAdd(&outdeg[s], 1u);
        atomicAdd(c ? &win[d] : &sin[d], 1u);
        if (weak && ((weak[e] != 0) != c))
            atomicOr(&flags[PK_EDGE_KIND], 1u);
    }
}

// ---- step 3: per-task limits, and the sources flagged for their list
__global__ void pk_degrees_kernel(const u8 *kinds, const u32 *outdeg, const u32 *sin, const u32 *win, u32 n,
                                  u32 *is_src, u32 *flags)
{
    u32 ns = 0;
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += grid_stride()) {
        const u32 od = outdeg[v], si = sin[v];
        if ((pk_cond(kinds[v]) && od == 0u) || od > 0xFFFFu || si > 0xFFFFu)
            atomicOr(&flags[PK_INVALID], 1u);
        const u32 f = (si == 0u && win[v] == 0u) ? 1u : 0u;
        is_src[v] = f;
        ns += f;
    }
    ns = __reduce_add_sync(kAll, ns);
    if ((threadIdx.x & 31) == 0 && ns)
        atomicAdd(&flags[PK_NSRC], ns);
}

// ---- exclusive scans of u32 counts (out-degrees, source flags, sort
// histograms): per-block sums, a scan of the sums, then each block's scan
// from its offset.  A block takes kScanChunk consecutive elements, each
// thread kScanPer consecutive ones.

// Exclusive scan of v over the block; *total gets the block's sum.
__device__ __forceinline__ u32 block_exclusive(u32 v, u32 *total)
{
    __shared__ u32 s_w[32];
    __shared__ u32 s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kAll, inc, o);
        if (lane >= o)
            inc += y;
    }
    if (lane == 31)
        s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        u32 t = lane < nw ? s_w[lane] : 0u;
        u32 ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(kAll, ti, o);
            if (lane >= o)
                ti += y;
        }
        if (lane < nw)
            s_w[lane] = ti - t;   // exclusive prefix of the warp sums
        if (lane == nw - 1)
            s_tot = ti;
    }
    __syncthreads();
    const u32 out = s_w[warp] + inc - v;
    const u32 tot = s_tot;
    __syncthreads();   // s_w and s_tot are reused by the next call
    *total = tot;
    return out;
}

__global__ void __launch_bounds__(kScanThreads) pk_scan_sums_kernel(const u32 *in, u32 len, u32 *sums)
{
    const u64 base = (u64)blockIdx.x * kScanChunk + (u64)threadIdx.x * kScanPer;
    u32 s = 0;
#pragma unroll
    for (u32 i = 0; i < kScanPer; ++i)
        if (base + i < len)
            s += in[base + i];
    u32 tot = 0;
    (void)block_exclusive(s, &tot);
    if (threadIdx.x == 0)
        sums[blockIdx.x] = tot;
}

// one block: exclusive scan of nsums block sums, in segments with a carry
__global__ void __launch_bounds__(kScanThreads) pk_scan_top_kernel(u32 *sums, u32 nsums)
{
    u32 carry = 0;
    for (u32 b = 0; b < nsums; b += kScanThreads) {
        const u32 i = b + threadIdx.x;
        const u32 v = i < nsums ? sums[i] : 0u;
        u32 tot = 0;
        const u32 ex = block_exclusive(v, &tot);
        if (i < nsums)
            sums[i] = carry + ex;
        carry += tot;
    }
}

// out[i] = offset of the block + exclusive prefix within it (out may be in)
__global__ void __launch_bounds__(kScanThreads) pk_scan_apply_kernel(const u32 *in, u32 len, const u32 *sums,
                                                                     u32 *out)
{
    const u64 base = (u64)blockIdx.x * kScanChunk + (u64)threadIdx.x * kScanPer;
    u32 v[kScanPer];
    u32 s = 0;
#pragma unroll
    for (u32 i = 0; i < kScanPer; ++i) {
        v[i] = base + i < len ? in[base + i] : 0u;
        s += v[i];
    }
    u32 tot = 0;
    u32 run = sums[blockIdx.x] + block_exclusive(s, &tot);
#pragma unroll
    for (u32 i = 0; i < kScanPer; ++i)
        if (base + i < len) {
            out[base + i] = run;
            run += v[i];
        }
}

// ---- step 4: one pass of the stable radix sort of (source, target) pairs
// by the source's digit at `shift`.  A block sorts kSortTile consecutive
// edges: warp w takes edges [w * 512, (w + 1) * 512) of the tile in rounds
// of 32, so that (warp, round, lane) order is the edges' order.

// hist[digit * ntiles + tile] = edges of the tile with that digit
__global__ void __launch_bounds__(256) pk_hist_kernel(const u32 *keys, u32 m, u32 shift, u32 ntiles, u32 *hist)
{
    __shared__ u32 cnt[256];
    cnt[threadIdx.x] = 0u;
    __syncthreads();
    const u64 base = (u64)blockIdx.x * kSortTile;
    for (u32 i = threadIdx.x; i < kSortTile; i += 256u) {
        const u64 e = base + i;
        if (e < m)
            atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(u64)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// hist scanned (digit-major): an edge goes to the offset of its digit in its
// tile + the edges of that digit before it in the tile
__global__ void __launch_bounds__(kSortWarps * 32) pk_sort_scatter_kernel(const u32 *kin, const u32 *vin, u32 *kout,
                                                                         u32 *vout, u32 m, u32 shift, u32 ntiles,
                                                                         const u32 *hist)
{
    __shared__ u32 s_off[256];
    __shared__ u32 s_cnt[kSortWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s_off[threadIdx.x] = hist[(u64)threadIdx.x * ntiles + blockIdx.x];
    for (u32 w = 0; w < kSortWarps; ++w)
        s_cnt[w][threadIdx.x] = 0u;
    __syncthreads();
    const u64 base = (u64)blockIdx.x * kSortTile + (u64)warp * (kSortRounds * 32u);
    // per edge: its digit (bits 16+) and its rank among the warp's edges of
    // that digit (bits 0-15, < 512)
    u32 pk[kSortRounds];
#pragma unroll
    for (u32 r = 0; r < kSortRounds; ++r) {
        const u64 e = base + r * 32u + (u32)lane;
        const bool ok = e < m;
        const u32 d = ok ? (kin[e] >> shift) & 255u : 256u;   // 256: no edge (a group of its own)
        const u32 peers = __match_any_sync(kAll, d);
        const u32 lower = peers & ((1u << lane) - 1u);
        const u32 before = ok ? s_cnt[warp][d] : 0u;
        __syncwarp();
        if (ok && lower == 0u)
            s_cnt[warp][d] = before + (u32)__popc(peers);
        __syncwarp();
        pk[r] = (d << 16) | (before + (u32)__popc(lower));
    }
    __syncthreads();
    {
        // per digit: where each warp's edges of it start, in warp order
        const u32 d = threadIdx.x;
        u32 run = 0;
        for (u32 w = 0; w < kSortWarps; ++w) {
            const u32 t = s_cnt[w][d];
            s_cnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (u32 r = 0; r < kSortRounds; ++r) {
        const u64 e = base + r * 32u + (u32)lane;
        if (e < m) {
            const u32 d = pk[r] >> 16;
            const u32 pos = s_off[d] + s_cnt[warp][d] + (pk[r] & 0xFFFFu);
            kout[pos] = kin[e];
            vout[pos] = vin[e];
        }
    }
}

// ---- step 5: the packed graph

// the 32-byte records: successor range, degrees, rounds | kind | argument,
// the task's id; join word = strong in-degree, count = digest = 0
__global__ void pk_records_kernel(const u8 *kinds, const u32 *params, const u32 *outdeg, const u32 *sin,
                                  const u32 *off, u32 n, u32 edge_base, NodeSlot *slots)
{
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += grid_stride()) {
        const u32 k = kinds[v], p = params[v];
        const u32 arg = k == TG_COND_LOOP ? (p >> 16) & 0xFFu : (k == TG_COND_CONST ? p >> 24 : 0u);
        uint4 *r = reinterpret_cast<uint4 *>(&slots[v]);
        r[0] = make_uint4(edge_base + off[v], outdeg[v] | (sin[v] << 16), (p & 0xFFFFu) | (k << 16) | (arg << 24), v);
        r[1] = make_uint4(sin[v], 0u, 0u, 0u);
    }
}

// successor ids in sorted (source, insertion) order; a strong edge to a task
// with no other strong in-edge carries the sole-predecessor bit
__global__ void pk_succ_kernel(const u32 *skey, const u32 *sval, const u8 *kinds, const u32 *sin, u32 m, u32 *out)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += grid_stride()) {
        const u32 d = sval[i];
        out[i] = d | ((!pk_cond(kinds[skey[i]]) && sin[d] == 1u) ? kSoleBit : 0u);
    }
}

// the sources in task order, at their scanned positions
__global__ void pk_sources_kernel(const u32 *is_src, const u32 *pos, u32 n, u32 *out)
{
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += grid_stride())
        if (is_src[v])
            out[pos[v]] = v;
}

__global__ void pk_fill_kernel(u32 *p, u32 count, u32 val)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += grid_stride())
        p[i] = val;
}

__global__ void pk_desc_kernel(GDesc *d, u32 seed, u32 node_off, u32 n, u32 src_off, u32 n_src, u32 exec_cap)
{
    GDesc g{};
    g.pe = 0;
    g.status = 0;
    g.seed = seed;
    g.node_off = node_off;
    g.n = n;
    g.src_off = src_off;
    g.n_src = n_src;
    g.exec_cap = exec_cap;
    g.ret = kEmpty32;
    g.acc = 0;
    *d = g;
}

u32 grid_for(u64 count)
{
    const u64 b = (count + 255u) / 256u;
    return (u32)(b == 0 ? 1 : (b > 148u * 16u ? 148u * 16u : b));
}

u32 scan_blocks(u64 len) { return (u32)((len + kScanChunk - 1) / kScanChunk); }

u32 sort_tiles(u32 m) { return (m + kSortTile - 1u) / kSortTile; }

cudaError_t scan_exclusive(const u32 *in, u32 len, u32 *out, u32 *sums, cudaStream_t st)
{
    if (len == 0)
        return cudaSuccess;
    const u32 nb = scan_blocks(len);
    pk_scan_sums_kernel<<<nb, kScanThreads, 0, st>>>(in, len, sums);
    pk_scan_top_kernel<<<1, kScanThreads, 0, st>>>(sums, nb);
    pk_scan_apply_kernel<<<nb, kScanThreads, 0, st>>>(in, len, sums, out);
    return cudaGetLastError();
}

size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

}  // namespace

size_t pack_scratch_bytes(u32 n, u32 m)
{
    const u64 nt = sort_tiles(m);
    const u64 nsums = (scan_blocks(n) > scan_blocks(256u * nt) ? scan_blocks(n) : scan_blocks(256u * nt)) + 1u;
    return align256(n) + align256(m) + align256((size_t)4 * n) + 4 * align256((size_t)4 * m) +
           6 * align256((size_t)4 * n) + 256 + align256((size_t)4 * 256 * nt) + align256((size_t)4 * nsums);
}

void pack_carve(char *base, u32 n, u32 m, PackBufs &b)
{
    char *p = base;
    auto take = [&](size_t bytes) {
        char *r = p;
        p += align256(bytes);
        return r;
    };
    b.kinds = (u8 *)take(n);
    b.weak = (u8 *)take(m);
    b.params = (u32 *)take((size_t)4 * n);
    b.src = (u32 *)take((size_t)4 * m);
    b.dst = (u32 *)take((size_t)4 * m);
    b.k1 = (u32 *)take((size_t)4 * m);
    b.v1 = (u32 *)take((size_t)4 * m);
    b.outdeg = (u32 *)take((size_t)4 * n);
    b.sin = (u32 *)take((size_t)4 * n);
    b.win = (u32 *)take((size_t)4 * n);
    b.is_src = (u32 *)take((size_t)4 * n);
    b.off = (u32 *)take((size_t)4 * n);
    b.srcpos = (u32 *)take((size_t)4 * n);
    b.flags = (u32 *)take(256);
    b.hist = (u32 *)take((size_t)4 * 256 * sort_tiles(m));
    b.sums = (u32 *)p;
}

cudaError_t pack_validate(const PackBufs &b, u32 n, u32 m, bool weak, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(b.flags, 0, PK_FLAGS * sizeof(u32), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b.outdeg, 0, (size_t)4 * n, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b.sin, 0, (size_t)4 * n, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b.win, 0, (size_t)4 * n, st);
    if (e != cudaSuccess)
        return e;
    pk_nodes_kernel<<<grid_for(n), 256, 0, st>>>(b.kinds, b.params, n, b.flags);
    if (m)
        pk_edges_kernel<<<grid_for(m), 256, 0, st>>>(b.kinds, b.src, b.dst, weak ? b.weak : nullptr, n, m, b.outdeg,
                                                     b.sin, b.win, b.flags);
    pk_degrees_kernel<<<grid_for(n), 256, 0, st>>>(b.kinds, b.outdeg, b.sin, b.win, n, b.is_src, b.flags);
    return cudaGetLastError();
}

cudaError_t pack_build(const PackBufs &b, u32 n, u32 m, const PackDest &d, cudaStream_t st)
{
    cudaError_t e = scan_exclusive(b.outdeg, n, b.off, b.sums, st);
    if (e != cudaSuccess)
        return e;
    pk_records_kernel<<<grid_for(n), 256, 0, st>>>(b.kinds, b.params, b.outdeg, b.sin, b.off, n, d.edge_base,
                                                   d.slots);
    // (source, target) pairs sorted by source, stably, 8 bits a pass over
    // the bits a task id of this graph uses
    u32 *ka = b.src, *va = b.dst, *kb = b.k1, *vb = b.v1;
    if (m && n > 1u) {
        const u32 bits = 32u - (u32)__builtin_clz(n - 1u);
        const u32 nt = sort_tiles(m);
        for (u32 shift = 0; shift < bits; shift += 8u) {
            pk_hist_kernel<<<nt, 256, 0, st>>>(ka, m, shift, nt, b.hist);
            if ((e = scan_exclusive(b.hist, 256u * nt, b.hist, b.sums, st)) != cudaSuccess)
                return e;
            pk_sort_scatter_kernel<<<nt, kSortWarps * 32, 0, st>>>(ka, va, kb, vb, m, shift, nt, b.hist);
            u32 *t = ka;
            ka = kb;
            kb = t;
            t = va;
            va = vb;
            vb = t;
        }
    }
    if (m)
        pk_succ_kernel<<<grid_for(m), 256, 0, st>>>(ka, va, b.kinds, b.sin, m, d.edges);
    if ((e = scan_exclusive(b.is_src, n, b.srcpos, b.sums, st)) != cudaSuccess)
        return e;
    pk_sources_kernel<<<grid_for(n), 256, 0, st>>>(b.is_src, b.srcpos, n, d.edges + m);
    pk_fill_kernel<<<grid_for(d.n_chunks), 256, 0, st>>>(d.chunk_gid, d.n_chunks, d.gid);
    pk_desc_kernel<<<1, 1, 0, st>>>(d.desc, d.seed, d.node_off, n, d.edge_base + m, d.n_src, d.exec_cap);
    return cudaGetLastError();
}

}  // namespace tg
