// FastFCA kernels specialised for M = 3 microphones, N = 2..8 sources.
#include "launch.cuh"

namespace ffca {

bool fast_ops_m3(int N, FastOps* o) {
  switch (N) {
    case 2: *o = make_fast_ops<3, 2>(); return true;
    case 3: *o = make_fast_ops<3, 3>(); return true;
    case 4: *o = make_fast_ops<3, 4>(); return true;
    case 5: *o = make_fast_ops<3, 5>(); return true;
    case 6: *o = make_fast_ops<3, 6>(); return true;
    case 7: *o = make_fast_ops<3, 7>(); return true;
    case 8: *o = make_fast_ops<3, 8>(); return true;
    default: return false;
  }
}

}  // namespace ffca
