// pass.cuh -- per-pass arguments that a captured launch sequence reads from
// device memory: the map count and the caller's buffers of this pass, so one
// CUDA graph serves every pass of a plan.
#pragma once

namespace drc {

struct PassSlot {
  int count;            // maps this pass (clamped by the kernels to the planned maximum)
  unsigned flags;       // DRC_F_ENCODE_INPUT / DRC_F_DECODE_OUTPUT of this pass
  const float *in;      // [count][7][H][W]
  float *out;           // [count][3][H][W]
  float *payload;       // [count][3], or nullptr
};

constexpr unsigned SLOT_ENCODE = 0x1u;  // same bits as the public flags
constexpr unsigned SLOT_DECODE = 0x2u;

}  // namespace drc
