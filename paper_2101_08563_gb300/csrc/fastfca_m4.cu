// FastFCA kernels specialised for M = 4 microphones, N = 2..4 sources (N = 5..8 are in
// fastfca_m4_hi.cu, so that the two halves compile in parallel).
#include "launch.cuh"

namespace ffca {

bool fast_ops_m4_hi(int N, FastOps* o);

bool fast_ops_m4(int N, FastOps* o) {
  switch (N) {
    case 2: *o = make_fast_ops<4, 2>(); return true;
    case 3: *o = make_fast_ops<4, 3>(); return true;
    case 4: *o = make_fast_ops<4, 4>(); return true;
    default: return fast_ops_m4_hi(N, o);
  }
}

}  // namespace ffca
