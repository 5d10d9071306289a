// TMA tensor maps for the tcgen05 GEMMs: operands are BF16 arrays viewed as
// [batch][rows][K] with 128-byte swizzle; out-of-range rows, columns and K read
// as zero.
#pragma once
#include "internal.cuh"
#include "tc_common.cuh"

namespace ea {

struct TmaMap {
  CUtensorMap map;
};
// Map over a bf16 array viewed as [nb][rows][K] with the given pitches (elements).
TmaMap make_tma_3d(const bf16* base, long long K, long long rows, long long nb, long long row_pitch,
                   long long batch_pitch, int box_rows);

}  // namespace ea
