// batch.cuh -- internal entry of the batched-region path for other parts of
// the library (the served request loop).
#pragma once

#include "common.cuh"

namespace accr {
// Plans and launches `nregions` regions (the accr_batch_reduce device path)
// on `stream`; variables go to the device addresses in the descriptors.
// tile_bytes > 0 cuts long regions into tiles of that size instead of the
// process-wide tiling (accr_batch_tiling); the split of a region still
// depends only on its own type and length.
int batch_launch_regions(const accr_region *regions, int64_t nregions, accr_stream_t stream, int64_t tile_bytes = 0);
}  // namespace accr
