// Layout of the reaction surrogate's parameters and normalisation, shared by
// the training code (bbx_mlp.cu) and the step kernel's inference.
#pragma once

#include "../../include/bbx.h"

namespace bbx {

// 8 -> 64 -> 64 -> 8, row-major weights, packed W1 b1 W2 b2 W3 b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + 64 * 8;
constexpr int kOffW2 = kOffB1 + 64;
constexpr int kOffB2 = kOffW2 + 64 * 64;
constexpr int kOffW3 = kOffB2 + 64;
constexpr int kOffB3 = kOffW3 + 8 * 64;
constexpr int kMlpParams = kOffB3 + 8;  // 5256

// normalisation: x = (s - mu_in) / sd_in, s' - s = y * sd_out + mu_out;
// envelope [lo, hi] of the training inputs (raw units)
constexpr int kNormMuIn = 0;
constexpr int kNormSdIn = 8;
constexpr int kNormMuOut = 16;
constexpr int kNormSdOut = 24;
constexpr int kNormLo = 32;
constexpr int kNormHi = 40;
constexpr int kNormSize = 48;

}  // namespace bbx

const float* bbx_mlp_device_params(const bbx_mlp* m);
const float* bbx_mlp_device_norm(const bbx_mlp* m);
