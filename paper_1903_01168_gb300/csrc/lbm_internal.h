// lbm_internal.h -- host helpers shared between the translation units of the
// library (not part of the C ABI).
#pragma once

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Validate a parameter set (message into err, 256 bytes).
lbm_status host_validate(int nx, int ny, const lbm_params *p, char *err);

// Fill a descriptor for a state buffer laid out as by lbm_create (densities
// region followed by deviations region).  Tensor maps are left zero.
void host_fill_desc(SimDesc &h, int nx, int ny, const lbm_params *p, void *state);

// Message returned by lbm_last_error(NULL) on this thread.
void host_set_global_error(const char *msg);

}  // namespace lbm
