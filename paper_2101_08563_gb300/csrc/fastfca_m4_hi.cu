// FastFCA kernels specialised for M = 4 microphones, N = 5..8 sources.
#include "launch.cuh"

namespace ffca {

bool fast_ops_m4_hi(int N, FastOps* o) {
  switch (N) {
    case 5: *o = make_fast_ops<4, 5>(); return true;
    case 6: *o = make_fast_ops<4, 6>(); return true;
    case 7: *o = make_fast_ops<4, 7>(); return true;
    case 8: *o = make_fast_ops<4, 8>(); return true;
    default: return false;
  }
}

}  // namespace ffca
