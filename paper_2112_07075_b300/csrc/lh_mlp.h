// Sizes of the learned-form MLP (per element: 3 previous accelerations at the
// (p+1)^3 = 64 nodes of a Q3 hexahedron x 3 components = 576 inputs, plus 10
// Jacobian features; 192 outputs = one acceleration correction per element DOF).
#pragma once

namespace lh {
namespace mlp {
constexpr int kIn = 586;      // 3 * 192 accelerations + 9 J entries + det J
constexpr int kInPad = 592;   // padded to a multiple of the MMA K step (16)
constexpr int kHid = 128;
constexpr int kOut = 192;
}  // namespace mlp
}  // namespace lh
