// FCA comparison-model kernels: M = 2..4 microphones, N = 2..8 sources.
#include "fca.cuh"

namespace ffca {

namespace {
template <int M>
bool fca_ops_m(int N, FcaOps* o) {
  switch (N) {
    case 2: *o = make_fca_ops<M, 2>(); return true;
    case 3: *o = make_fca_ops<M, 3>(); return true;
    case 4: *o = make_fca_ops<M, 4>(); return true;
    case 5: *o = make_fca_ops<M, 5>(); return true;
    case 6: *o = make_fca_ops<M, 6>(); return true;
    case 7: *o = make_fca_ops<M, 7>(); return true;
    case 8: *o = make_fca_ops<M, 8>(); return true;
    default: return false;
  }
}
}  // namespace

bool fca_ops(int M, int N, FcaOps* o) {
  switch (M) {
    case 2: return fca_ops_m<2>(N, o);
    case 3: return fca_ops_m<3>(N, o);
    case 4: return fca_ops_m<4>(N, o);
    default: return false;
  }
}

}  // namespace ffca
