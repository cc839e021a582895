// Cluster-kernel FastFCA and FastMNMF ops (large bins) for M = 6..8 microphones, any N <= 16.
#include "fastmnmf_cluster.cuh"
#include "launch.cuh"

namespace ffca {

bool cluster_ops_lo(int M, int N, int T, FastOps* o);

bool cluster_ops(int M, int N, int T, FastOps* o) {
  int C = 0;
  size_t smem = 0;
  switch (M) {
    case 6: if (!cluster_shape<6>(T, N, &C, &smem)) return false; *o = make_cluster_ops<6>(); break;
    case 7: if (!cluster_shape<7>(T, N, &C, &smem)) return false; *o = make_cluster_ops<7>(); break;
    case 8: if (!cluster_shape<8>(T, N, &C, &smem)) return false; *o = make_cluster_ops<8>(); break;
    default: return cluster_ops_lo(M, N, T, o);
  }
  o->max_T = T;
  o->cluster_c = C;
  prefer_sm_kernel(M, N, T, o);
  return true;
}

bool mnmf_cluster_ops_lo(int M, int N, int T, MnmfOps* o);

bool mnmf_cluster_ops(int M, int N, int T, MnmfOps* o) {
  switch (M) {
    case 6: return mnmf_cluster_ops_m<6>(N, T, o);
    case 7: return mnmf_cluster_ops_m<7>(N, T, o);
    case 8: return mnmf_cluster_ops_m<8>(N, T, o);
    default: return mnmf_cluster_ops_lo(M, N, T, o);
  }
}

}  // namespace ffca
