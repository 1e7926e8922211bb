// Exclusive prefix sums on the device (three launches: block scans, scan of block totals,
// offset add).  Used by the neighbour build; not on the recurrence path.
#pragma once
#include "common.cuh"

namespace tbk {

// out[0..n] = exclusive prefix sums of in[0..n-1] (out[n] = total).  `tmp` must hold
// scan_tmp_elems(n) int64.
size_t scan_tmp_elems(int64_t n);
void exclusive_scan_i32(tbk_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, int64_t* tmp);

}  // namespace tbk
