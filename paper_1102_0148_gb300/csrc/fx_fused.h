// Host interface of the fused F/X-engine: one persistent launch that
// transforms and cross-multiplies a whole run of device-resident input for
// the K = 512, FP32-mode correlator with up to 44 antennas.
#pragma once

#include <string>

#include "corr_internal.h"

namespace gbcorr {

constexpr int kFxMaxN = 44;          // antennas the fused kernel's shared memory serves
constexpr int kFxMaxBlocks = 8192;   // 32-frame blocks per launch (262144 frames)

// One run of consecutive frames of device input: [frames][N][256] bytes.
struct FxSegment {
    const uint8_t* in;
    int64_t frames;
};

struct FxPlan;

// True when the fused kernel serves this geometry and workspace type.
bool fx_supported(int N, int K, int spec_type);
// Ring, counters and block tables of the fused kernel for N antennas.
int fx_plan_create(FxPlan** out, int N, std::string& err);
void fx_plan_destroy(FxPlan* p);
// Blocks that `segs` occupy: each segment is padded to whole 32-frame blocks.
int64_t fx_blocks(const FxSegment* segs, int nseg);
// Queue one launch over the segments (at most kFxMaxBlocks blocks) on `st`,
// adding V of every channel into acc ([256][P] FP64).  split: [N]
// two-plane pre-scales; corr: [N][256] corrections or nullptr.  A bounded
// device-side wait that gives up records a status in `status` (the handle's
// CORR_ETIMEOUT path).  test_withhold: the first chunk's completion count is
// never reached (the failure-path test hook; wait_limit in seconds).
int fx_launch(FxPlan* p, const FxSegment* segs, int nseg, const float2* twiddle,
              const float* split, const float2* corr, double2* acc, int* status, cudaStream_t st,
              std::string& err);
int fx_test_withhold(FxPlan* p, double wait_limit_s, std::string& err);

}  // namespace gbcorr
