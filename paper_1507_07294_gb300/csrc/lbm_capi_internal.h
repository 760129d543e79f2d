// Accessors of lbm_ctx for the batch engine (lbm_batch.cu); lbm_ctx itself is private
// to lbm_capi.cu.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

int ctx_storage(const lbm_ctx* c);
// Whether the run can join a batch (pattern AB, coupled mode, default model variant,
// initialised); if not, *why says why.
bool ctx_batchable(const lbm_ctx* c, std::string* why);
bool ctx_have_prev(const lbm_ctx* c);
cudaStream_t ctx_stream(const lbm_ctx* c);
void ctx_describe(const lbm_ctx* c, Geometry* geo, Physics* ph, float** state0, float** state1,
                  float** phi, float** mu, int* parity);
// Book-keeping after the batch advanced the run by n steps.
void ctx_advance(lbm_ctx* c, int n);

}  // namespace lbm
