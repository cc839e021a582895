// Learned initialiser of FastFCA (not in the paper): GPU mixture generator, features, a small
// MLP trained with BF16 tensor-core products accumulated in FP32, and the head that turns the
// network output into a starting point (W, L, H) of Algorithm 1.  The definitions follow the
// FP64 reference used by the tests (features, network, conv over t, scale- and
// permutation-free loss); see the header of the C ABI for the interface.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "philox.cuh"

namespace ffca {
namespace learn {

constexpr int kDin = 16;          // feature length
constexpr int kHidden = 256;
constexpr int kOutPad = 40;       // network output columns (2M^2 + MN + N <= 40 for M=3, N=5)
constexpr int kConvK = 9;         // taps of the 1-D conv over t
constexpr int kMaxN = 5;
constexpr int kMaxM = 3;

}  // namespace learn
}  // namespace ffca
