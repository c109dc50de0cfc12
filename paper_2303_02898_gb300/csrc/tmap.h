// tmap.h -- tensor maps (TMA descriptors) for the tensor-core kernels (host).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace mem_host {

// A 2D FP32 row-major tensor of `rows` rows and `cols` columns (cols
// innermost, row stride cols * 4 bytes), read in boxes of box_rows x box_cols
// elements into shared memory with the 128-byte swizzle (box_cols * 4 <= 128).
// The encoder comes from the driver through the runtime's entry-point query
// (no link against the driver library).  MEM_ECUDA if it is unavailable or
// rejects the arguments.
int encode_tmap_2d_f32(CUtensorMap *out, const void *base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                       uint32_t box_rows);

}  // namespace mem_host
