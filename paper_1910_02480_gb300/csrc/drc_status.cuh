// drc_status.cuh -- status codes that device code latches into a context's
// status word; the values are those of drc_status in include/drc.h.
#pragma once

namespace drc {
constexpr int ERR_TIMEOUT = 5;  // DRC_ERR_TIMEOUT
}  // namespace drc
