// batch.cuh -- internal entries of the batched-region path for other parts of
// the library (the served request loop, the row nest's split-row path).
#pragma once

#include "common.cuh"

namespace accr {
// Plans and launches `nregions` regions (the accr_batch_reduce device path)
// on `stream`; variables go to the device addresses in the descriptors.
// tile_bytes > 0 cuts long regions into tiles of that size instead of the
// process-wide tiling (accr_batch_tiling); the split of a region still
// depends only on its own type and length.
int batch_launch_regions(const accr_region *regions, int64_t nregions, accr_stream_t stream, int64_t tile_bytes = 0);
// The rows of a row-major matrix as regions of one batch (row r: cols
// elements from A + r * ld; variable r of clause c at cl[c].out + r), cut into
// tiles of tile_bytes (the row nest's split-row path).
int batch_launch_rows(const void *A, int64_t rows, int64_t cols, int64_t ld, int in_type, const ClauseDev *cl, int nc,
                      int64_t tile_bytes, accr_stream_t stream);
}  // namespace accr
