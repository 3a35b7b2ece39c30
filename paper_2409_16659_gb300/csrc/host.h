// host.h -- host-side helpers shared by the single-lattice handle
// (mlswlbm.cu) and batches (batch.cu). Not part of the C ABI.
#pragma once

#include <cuda.h>

#include "../../include/mlswlbm.h"
#include "kernels.h"

namespace mlsw_host {

int Qof(int lattice);

// Validates one lattice (parameters, heights, create-time stability check)
// and fills its device parameters: kp with the padded layout, ghost tables
// and rest-population shift H (the median of each layer of h_init), and sh.
// MLSW_OK or an MLSW_ERR_* code.
int prepare_instance(const mlsw_params& p, const float* h_init, mlsw::KParams& kp,
                     mlsw::KShift& sh);

// 3-D tensor map of a population buffer: dims (pitch, rows, nplanes), box
// (box_cols, box_rows, nplanes) floats.
bool make_tile_map(CUtensorMap* m, float* base, const mlsw::Layout& L, int nplanes, int box_cols,
                   int box_rows);

// The device address of a page-locked host buffer, or nullptr.
const void* mapped_host_ptr(const void* p);

}  // namespace mlsw_host
