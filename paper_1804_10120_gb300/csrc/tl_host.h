// tl_host.h -- host-side helpers shared by the C-ABI translation units (not part of the ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tl.h"

namespace tl {

tl_status fail(tl_status s, const char *fmt, ...);
tl_status cuda_fail(cudaError_t e, const char *what);

constexpr int kMaxDevices = 64;
struct DeviceInfo {
    bool ready = false;
    bool supported = false;
    int sms = 0;
    int fwd_f64_blocks = 0, fwd_f32_blocks = 0, fwd_ff_blocks = 0, bwd_f64_blocks = 0, bwd_ff_blocks = 0;
    int fwdbwd_f64_blocks = 0, fwdbwd_ff_blocks = 0;
    char name[256] = {0};
};
// Facts about the current device (sm_103 check, SM count, occupancies), queried once per device.
tl_status device_info(const DeviceInfo **out);

size_t elem_size(tl_dtype t);
bool dtype_ok(int t);

struct Range {
    uintptr_t lo, hi;
    bool write;
    const char *name;
    int index, grid;
};
tl_status collect_ranges(std::vector<Range> &rs, const void *const *tabs[], const int counts[], const bool writes[],
                         const bool nullable[], const char *const names[], int ntabs, int64_t n, size_t esz, int grid);
tl_status check_overlaps(std::vector<Range> &rs);

}  // namespace tl
