// FastFCA kernels specialised for M = 4 microphones, N = 2..8 sources.
#include "launch.cuh"

namespace ffca {

bool fast_ops_m4(int N, FastOps* o) {
  switch (N) {
    case 2: *o = make_fast_ops<4, 2>(); return true;
    case 3: *o = make_fast_ops<4, 3>(); return true;
    case 4: *o = make_fast_ops<4, 4>(); return true;
    case 5: *o = make_fast_ops<4, 5>(); return true;
    case 6: *o = make_fast_ops<4, 6>(); return true;
    case 7: *o = make_fast_ops<4, 7>(); return true;
    case 8: *o = make_fast_ops<4, 8>(); return true;
    default: return false;
  }
}

}  // namespace ffca
