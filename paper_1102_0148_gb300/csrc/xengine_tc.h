// Host interface of the tensor-core (tcgen05) X-engine.
#pragma once

#include <string>

#include "corr_internal.h"

namespace gbcorr {

struct TcPlan;

// Prepare a plan for N antennas and C channels of workspace type spec_type.
int tc_plan_create(TcPlan** out, int N, int C, int spec_type, std::string& err);
// (Re)bind the plan to a workspace of `cap` frames per row.
int tc_plan_update(TcPlan* p, void* spec, int64_t cap, int N, int C, int spec_type, std::string& err);
// Run the X-engine over S_pad frames.  When the pass is one work item per
// channel the epilogue adds V straight into the FP64 accumulator `acc`
// ([C][P]) and *direct is set; otherwise it writes tc_num_partials() partial
// blocks of [C][P] complex64 to `partial` for the reduction kernel.
int tc_run(TcPlan* p, int64_t S_pad, float2* partial, double2* acc, const float* scale,
           int* status, cudaStream_t st, std::string& err, bool* direct);
int tc_num_partials(const TcPlan* p, int64_t S_pad);
void tc_plan_destroy(TcPlan* p);

}  // namespace gbcorr
