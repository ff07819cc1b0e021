// hd_contrast.h -- host-side links between the contrast stretch (hd_contrast.cu)
// and the rest of the API (hd_api.cu).
#pragma once

namespace hd {

// Reads and clears the contrast kernel's device error word; returns cudaError_t.
int read_and_clear_contrast_error(unsigned int *out);

// Polls a bounded device-side wait makes before it gives up (hd_set_spin_limit).
unsigned long long spin_limit_polls();

}  // namespace hd
