// tg_result.cu -- read-back of a graph's results (tg_result_copy).
//
// A task record is 32 bytes, of which the caller wants the execution count
// and the digest (8 bytes); the outputs live in their own array.  Copying
// whole records to the host moves four times the bytes it needs, so the
// count and digest of every task are first packed on the device into one
// 64-bit word each, and only those words cross to the host.
#include "../../include/tg.h"
#include "tg_internal.h"

namespace tg {
namespace {

// dst[v] = digest (hi 32) | execution count without the in-flight and
// waiting bits (lo 32) of task node_off + v.
__global__ void result_gather_kernel(const NodeSlot *slots, u32 node_off, u32 n, u64 *dst)
{
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint2 s = __ldcg(reinterpret_cast<const uint2 *>(&slots[node_off + v].cnt));
        dst[v] = ((u64)s.y << 32) | (u64)(s.x & ~(kInflight | kAwait));
    }
}

}  // namespace

cudaError_t launch_result_gather(const NodeSlot *slots, u32 node_off, u32 n, u64 *dst, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    const u32 blocks = min((n + 255u) / 256u, 148u * 8u);
    result_gather_kernel<<<blocks, 256, 0, st>>>(slots, node_off, n, dst);
    return cudaGetLastError();
}

}  // namespace tg
