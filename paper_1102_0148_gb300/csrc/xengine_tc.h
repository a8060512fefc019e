// Host interface of the tensor-core (tcgen05) X-engine.
#pragma once

#include <string>

#include "corr_internal.h"

namespace gbcorr {

constexpr int kMaxTcModes = 4;

struct TcPlan;

// What one mode of a tensor-core launch reads and writes.
struct TcRun {
    int64_t S_pad;            // frames in the workspace pass (multiple of 128)
    float2* partial;          // [max_split][C][P] FP32 partials (split items; slot 0 holds
                              // a multi-block mode's whole pass result)
    double2* acc;             // [C][P] FP64 accumulator
    const float* scale;       // [N][C] pre-cast scales (FP16 / FP8), else nullptr
    const float* split;       // [N] two-plane pre-scales sigma_i (FP32 mode), else nullptr
    int* status;              // device status word (bounded waits)
    int n_split;              // out: partial slots the reduction adds (when !direct)
    bool direct;              // out: accumulated into acc in the kernel (single block)
};

// Prepare a plan for N antennas and C channels of workspace type spec_type.
int tc_plan_create(TcPlan** out, int N, int C, int spec_type, std::string& err);
// (Re)bind the plan to a workspace of `cap` frames per row.
int tc_plan_update(TcPlan* p, void* spec, int64_t cap, int N, int C, int spec_type, std::string& err);
// Tile choices: TMEM accumulation window (spectra, 0 = default), pipeline
// stages (0 = as many as shared memory holds, up to 8), ranges per channel
// of a pass (0 = the planner's choice) and k-tiles per stage (0 = automatic).
int tc_set_tiles(TcPlan* p, int window, int stages, int split, int atoms, std::string& err);
// One persistent launch over the passes of n plans sharing a precision.
// Modes whose run reports direct = false need the reduction of their
// n_split partial blocks into acc.
int tc_launch(TcPlan* const* plans, int n, TcRun* runs, cudaStream_t st, std::string& err);
// Test hook: the next launch's CTA 0 skips the copy of its first k-tile, so
// its MMA thread's bounded wait expires after wait_limit_s.
int tc_test_withhold(TcPlan* p, double wait_limit_s, std::string& err);
// Clear the split arrival counters (after an aborted launch).
int tc_reset(TcPlan* p);
void tc_plan_destroy(TcPlan* p);

}  // namespace gbcorr
