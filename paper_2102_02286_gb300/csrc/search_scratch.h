// Library-internal entry of the search in caller scratch (search.cu), used by
// the serving loop (server.cu) to run launches in blocks of its device pool.
#pragma once

#include "hicops_internal.h"

namespace hicops {

// A search whose scratch is caller memory, with the launch shape given
// (hicops_search_scratch takes the index's own).  scratch_bytes is what such
// a search of n spectra takes; the device's SM count must already be known
// (any check of a batch, or hicops_search_scratch_bytes, finds it).
uint64_t scratch_bytes(const hicops_index* idx, const hicops_search_config& cfg, uint32_t n);
hicops_status search_in_scratch(hicops_index* idx, const hicops_batch* b, const hicops_search_config& cfg,
                                void* scratch, uint64_t bytes, hicops_psm* out_psm, uint32_t* out_hist,
                                uint32_t* out_nscored);

}  // namespace hicops
