// Test hook for failure detection: one warp runs the library's two bounded
// look-back waits (chunk_prefix, used by the compaction and the splat and
// pair scans; lookback_walk, used by the radix passes, through
// lookback_prefix) as chunk/tile 1 against a word 0 that nothing ever
// publishes, with a small poll limit. Each wait gives up after max_polls
// polls, latches
// kStatusTimeout into the workspace's status word and returns, so the host
// reads S3R_ERR_TIMEOUT from the next s3r_sync_status and the context stays
// usable. The hook writes four words at the end of the look-back array,
// tagged with kStageProbe, which no pass uses.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

__global__ void __launch_bounds__(32) k_wait_probe(unsigned long long* words, uint32_t* ctr,
                                                   int max_polls) {
  __shared__ uint32_t s_red[1];
  const uint32_t tag = stage_tag(ctr[kCtrEpoch], kStageProbe);
  // words[0] and words[2]: the predecessors that never publish
  if (threadIdx.x == 0) {
    st_relaxed(words, 0ull);
    st_relaxed(words + 2, 0ull);
  }
  __syncthreads();
  chunk_prefix<1>(words, 1, tag, ctr, s_red, max_polls);            // reads words[0]
  if (threadIdx.x == 0) lookback_prefix(words + 2, 1, 1, tag, 1u, ctr, max_polls);   // words[3]
}

}  // namespace

cudaError_t launch_wait_probe(s3r_workspace* ws, int max_polls, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(ws->lookback + ws->lookback_words - 4, ws->ctr, max_polls);
  return cudaGetLastError();
}

}  // namespace s3r
