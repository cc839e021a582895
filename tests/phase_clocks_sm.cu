// Measurement program (not part of the library, not run by pytest): the phase clocks of
// fastfca_em_sm_kernel<8> on one full wave (F = 152 frequencies, one per SM) of the large
// shape (M = 8, N = 12, T frames, default 4000), from a build of the kernel with
// -DFFCA_PHASE_CLOCKS, which makes thread 0 of frequency 0 stamp clock64() at each phase
// boundary of the first 8 iterations.  Synthetic input: x ~ CN(0, 1), W = I, L = 1, H uniform.
// Prints the launch time and the cycles of each phase (pass A, Q, inverses, IP columns, U,
// n-loop) for iterations 1 and 2.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -DFFCA_PHASE_CLOCKS -I include \
//        tests/phase_clocks_sm.cu -o phase_clocks_sm && ./phase_clocks_sm 4000 152
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <random>
#include "../paper_2101_08563_gb300/csrc/fastfca_em_sm.cuh"
using namespace ffca;
namespace ffca {
// host-side settings the library keeps in fastfca_sm.cu; unused by this program's launch
int large_bin_kernel_choice() { return 0; }
int cluster_wait_limit() { return 0; }
}
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e_), __LINE__); return 1; } } while (0)
int main(int argc, char** argv) {
  const int M = 8, N = 12, T = argc > 1 ? atoi(argv[1]) : 4000, F = argc > 2 ? atoi(argv[2]) : 152, iters = 4;
  std::mt19937 g(1);
  std::normal_distribution<float> nd(0.f, 1.f);
  std::uniform_real_distribution<float> ud(0.5f, 1.5f);
  std::vector<float2> x((size_t)F * T * M);
  for (auto& z : x) z = make_float2(nd(g), nd(g));
  std::vector<double2> P((size_t)F * M * M, make_double2(0, 0));
  for (int f = 0; f < F; ++f) for (int m = 0; m < M; ++m) P[(size_t)f * M * M + m * M + m] = make_double2(1, 0);
  std::vector<float> lam((size_t)F * M * N, 1.f), v((size_t)F * N * T);
  for (auto& a : v) a = ud(g) * (2.0f / N);
  float2* dx; double2* dP; float *dl, *dv; double2* dB; double* ddet; int* derr; double* dll; long long* dclk;
  CK(cudaMalloc(&dx, x.size() * 8)); CK(cudaMalloc(&dP, P.size() * 16)); CK(cudaMalloc(&dl, lam.size() * 4));
  CK(cudaMalloc(&dv, v.size() * 4)); CK(cudaMalloc(&dB, (size_t)F * M * M * 16)); CK(cudaMalloc(&ddet, (size_t)F * 16));
  CK(cudaMalloc(&derr, 4)); CK(cudaMalloc(&dll, (size_t)F * iters * 8)); CK(cudaMalloc(&dclk, 8 * 32 * 8));
  CK(cudaMemcpy(dx, x.data(), x.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemset(derr, 0, 4)); CK(cudaMemset(dclk, 0, 8 * 32 * 8));
  EmArgs a{};
  a.x = dx; a.P = dP; a.lam = dl; a.v = dv; a.ll_hist = dll; a.ll_last = nullptr; a.Bst = dB; a.detst = ddet;
  a.b_valid = 0; a.err = derr; a.F = F; a.T = T; a.n_iter = iters; a.ll_stride = iters; a.N = N; a.clocks = dclk;
  const size_t smem = SmSmem<M>::bytes;
  CK(cudaFuncSetAttribute(fastfca_em_sm_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float best = 1e9;
  for (int rep = 0; rep < 3; ++rep) {
    CK(cudaMemcpy(dP, P.data(), P.size() * 16, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dl, lam.data(), lam.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dv, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
    cudaEventRecord(e0);
    fastfca_em_sm_kernel<M><<<F, kSThreads, smem>>>(a);
    CK(cudaGetLastError());
    cudaEventRecord(e1);
    CK(cudaDeviceSynchronize());
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  int err; CK(cudaMemcpy(&err, derr, 4, cudaMemcpyDeviceToHost));
  std::vector<long long> clk(8 * 32); CK(cudaMemcpy(clk.data(), dclk, clk.size() * 8, cudaMemcpyDeviceToHost));
  printf("T=%d F=%d iters=%d: launch %.3f ms = %.1f us per iteration, err bits %d\n", T, F, iters, best, best * 1e3 / iters, err);
  const char* names[] = {"pass A", "Q pass + reduce", "inverses", "columns + sync", "U pass"};
  for (int it = 1; it < 3; ++it) {
    long long* c = &clk[it * 32];
    printf("iteration %d (cycles):", it);
    for (int s = 0; s < 5; ++s) printf(" %s %lld |", names[s], c[s + 1] - c[s]);
    long long nl = c[6 + N - 1] - c[5];
    printf(" n-loop %lld (per source %lld) | total %lld\n", nl, nl / N, clk[(it + 1) * 32] - c[0]);
  }
  return 0;
}
