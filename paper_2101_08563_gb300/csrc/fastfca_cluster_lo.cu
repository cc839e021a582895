// Cluster-kernel FastFCA and FastMNMF ops (large bins) for M = 2..5 microphones, any N <= 16.
#include "fastmnmf_cluster.cuh"
#include "launch.cuh"

namespace ffca {

bool cluster_ops_lo(int M, int N, int T, FastOps* o) {
  int C = 0;
  size_t smem = 0;
  switch (M) {
    case 2: if (!cluster_shape<2>(T, N, &C, &smem)) return false; *o = make_cluster_ops<2>(); break;
    case 3: if (!cluster_shape<3>(T, N, &C, &smem)) return false; *o = make_cluster_ops<3>(); break;
    case 4: if (!cluster_shape<4>(T, N, &C, &smem)) return false; *o = make_cluster_ops<4>(); break;
    case 5: if (!cluster_shape<5>(T, N, &C, &smem)) return false; *o = make_cluster_ops<5>(); break;
    default: return false;
  }
  o->max_T = T;
  o->cluster_c = C;
  prefer_sm_kernel(M, N, T, o);
  return true;
}

bool mnmf_cluster_ops_lo(int M, int N, int T, MnmfOps* o) {
  switch (M) {
    case 2: return mnmf_cluster_ops_m<2>(N, T, o);
    case 3: return mnmf_cluster_ops_m<3>(N, T, o);
    case 4: return mnmf_cluster_ops_m<4>(N, T, o);
    case 5: return mnmf_cluster_ops_m<5>(N, T, o);
    default: return false;
  }
}

}  // namespace ffca
