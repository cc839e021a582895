// FastMNMF kernels for M = 4 microphones, N = 2..8 sources, K = 1..16 bases per source.
#include "fastmnmf.cuh"

namespace ffca {
bool mnmf_ops_m4(int N, MnmfOps* o) { return mnmf_ops_for_m<4>(N, o); }
}  // namespace ffca
