// One-SM IP+EM kernels (fastfca_em_sm.cuh) for M = 5..8 microphones, and the host switches that
// tests use to run either large-bin kernel on one shape and to make a cluster exchange time out.
#include <atomic>

#include "../../include/fastfca.h"
#include "launch.cuh"

namespace ffca {

namespace {
std::atomic<int> g_large_bin_kernel{0};
std::atomic<int> g_cluster_wait_limit{0};
}

int large_bin_kernel_choice() { return g_large_bin_kernel.load(); }
int cluster_wait_limit() { return g_cluster_wait_limit.load(); }

EmLaunch sm_em_launcher(int M) {
  switch (M) {
    case 5: return &launch_em_sm<5>;
    case 6: return &launch_em_sm<6>;
    case 7: return &launch_em_sm<7>;
    case 8: return &launch_em_sm<8>;
    default: return nullptr;
  }
}

}  // namespace ffca

extern "C" void fastfca_debug_large_bin_kernel(int32_t which) {
  if (which >= 0 && which <= 2) ffca::g_large_bin_kernel.store(which);
}

extern "C" void fastfca_debug_cluster_wait_limit(int32_t spins) {
  ffca::g_cluster_wait_limit.store(spins > 0 ? spins : 0);
}
