// FastMNMF kernels for M = 3 microphones, N = 2..8 sources, K = 1..16 bases per source.
#include "fastmnmf.cuh"

namespace ffca {
bool mnmf_ops_m3(int N, MnmfOps* o) { return mnmf_ops_for_m<3>(N, o); }
}  // namespace ffca
