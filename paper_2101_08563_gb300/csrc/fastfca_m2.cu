// FastFCA kernels specialised for M = 2 microphones, N = 2..8 sources.
#include "launch.cuh"

namespace ffca {

bool fast_ops_m2(int N, FastOps* o) {
  switch (N) {
    case 2: *o = make_fast_ops<2, 2>(); return true;
    case 3: *o = make_fast_ops<2, 3>(); return true;
    case 4: *o = make_fast_ops<2, 4>(); return true;
    case 5: *o = make_fast_ops<2, 5>(); return true;
    case 6: *o = make_fast_ops<2, 6>(); return true;
    case 7: *o = make_fast_ops<2, 7>(); return true;
    case 8: *o = make_fast_ops<2, 8>(); return true;
    default: return false;
  }
}

}  // namespace ffca
