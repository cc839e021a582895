// Host-side check of the launch geometry the library computes, for every shape it accepts:
// threads per CTA, frames per thread and the shared memory each kernel asks for, against the
// GB300 limits (227 KB of dynamic shared memory per CTA, 48 KB of static, 1024 threads,
// clusters of at most 8, 512 tensor-memory columns per SM).  It includes the library's own launch headers and calls their
// host functions; it makes no CUDA call, so it runs without a GPU.  Prints "ok" or the first
// violation (and exits 1).
#include <cstdio>
#include <cstdlib>

#include "../paper_2101_08563_gb300/csrc/fca.cuh"
#include "../paper_2101_08563_gb300/csrc/launch.cuh"

using namespace ffca;

namespace {

constexpr size_t kDynMax = 227 * 1024;
constexpr size_t kStaticMax = 48 * 1024;
int failures = 0;

void fail(const char* what, int M, int N, int T, size_t value) {
  if (failures++ < 10) std::printf("FAIL %s: M=%d N=%d T=%d value=%zu\n", what, M, N, T, value);
}

// frequency-resident IP+EM kernel: T <= kMaxThreads * kSlots
template <int M, int N>
void check_em() {
  for (int T = 1; T <= kMaxThreads * kSlots; ++T) {
    const int th = em_threads(T);
    if (th % 32 || th > kMaxThreads || th * kSlots < T) fail("em threads", M, N, T, th);
    const size_t b = EmSmem<M, N>::bytes(th);
    if (b > kDynMax) fail("em smem", M, N, T, b);
  }
}

// full-rank FCA kernel (EM and MM): T <= kFcaMaxThreads * kFcaSlots
template <int M, int N, bool MM>
void check_fca() {
  for (int T = 1; T <= kFcaMaxThreads * kFcaSlots; ++T) {
    const int th = fca_threads(T);
    if (th % 32 || th > kFcaMaxThreads || th * kFcaSlots < T) fail("fca threads", M, N, T, th);
    const size_t b = FcaSmem<M, N, MM>::bytes(th);
    if (b > kDynMax) fail("fca smem", M, N, T, b);
  }
}

// frequency-resident Wiener filter: its image staging buffer is static shared memory
template <int M, int N>
void check_mwf() {
  constexpr int FSn = mwf_frame_stride(N, M);
  const size_t b = sizeof(float4) * ((kMwfThreads * FSn + 1) / 2 + 1) + sizeof(float2) * 2 * M * M +
                   sizeof(float) * M * N;
  if (FSn < N * M || ((N * M) % 2 == 0 && FSn % 2)) fail("mwf frame stride", M, N, 0, FSn);
  if (b > kStaticMax) fail("mwf static smem", M, N, 0, b);
}

// cluster kernel (runtime N <= kCMaxN) and the wide filter, for every T a cluster takes
template <int M>
void check_cluster() {
  for (int N = 1; N <= kCMaxN; ++N) {
    int accepted = 0;
    for (int T = 1; T <= 65536; ++T) {
      int C = 0;
      size_t smem = 0;
      if (!cluster_shape<M>(T, N, &C, &smem)) continue;
      ++accepted;
      const int Tc = (T + C - 1) / C;
      if (C != 1 && C != 2 && C != 4 && C != 8) fail("cluster size", M, N, T, C);
      if ((C - 1) * Tc >= T) fail("cluster CTA without frames", M, N, T, C);
      if (smem > kDynMax || smem != ClusterSmem<M>::bytes(N, Tc)) fail("cluster smem", M, N, T, smem);
    }
    if (accepted < 4000) fail("cluster accepts fewer than 4000 frames", M, N, accepted, accepted);
    // tiled filter: P threads per frame hold R rows each, covering the M rows, a whole number
    // of frames per warp; shared memory of one CTA, 16-byte alignment of every region and staged
    // frame (bulk copies), staged frames in odd 16-byte strides (conflict-free 16-byte stores)
    const MwfTileLayout L = mwf_tile_layout(M, N);
    if (mwf_tile_smem(M, N) > kDynMax) fail("tile filter smem", M, N, 0, mwf_tile_smem(M, N));
    if (L.k % 16 || L.wc % 16 || L.lt % 16 || L.h % 16 || L.out % 16 || L.total % 16)
      fail("tile filter region alignment", M, N, 0, L.total);
    if (mwf_tile_p(M) * mwf_tile_r(M) < M || (mwf_tile_p(M) - 1) * mwf_tile_r(M) >= M || 32 % mwf_tile_p(M) ||
        mwf_tile_frames(M) * mwf_tile_p(M) != 32)
      fail("tile filter threads per frame", M, N, mwf_tile_p(M), mwf_tile_r(M));
    // 16-byte vector accesses: every row segment a thread reads or writes starts on 16 bytes
    if (mwf_tile_vec(M))
      for (int qq = 0; qq < mwf_tile_p(M); ++qq)
        for (int a = 0; a < M; ++a)
          for (int n = 0; n < N; ++n)
            if ((a * M + qq * mwf_tile_r(M)) % 2 || ((n * M + a) * M + qq * mwf_tile_r(M)) % 2 ||
                (n * M + qq * mwf_tile_r(M)) % 2 || mwf_tile_r(M) % 2)
              fail("tile filter vector alignment", M, N, a, qq);
    const int FB = mwf_tile_frame_bytes(N, M);
    if (FB % 16 || (FB / 16) % 2 == 0 || FB < N * M * 8) fail("tile filter frame stride", M, N, 0, FB);
    if (L.wc - L.k < N * M * M * 8 || L.lt - L.wc < M * M * 8 || L.h - L.lt < kMwfWMaxN * M * 4 ||
        L.out - L.h < kMwfWMaxN * mwf_tile_frames(M) * 4)
      fail("tile filter region size", M, N, 0, L.total);
  }
  if (kCThreads > 1024 || kCThreads % 32) fail("cluster threads", M, 0, 0, kCThreads);
}

// one-SM IP+EM kernel: T <= kSMaxT frames, kSThreads threads, every thread's frames inside
// its kSSlots TMEM slots, every TMEM column it touches inside the kSCols allocated, 1/sigma^2
// and r rows inside the shared array, one CTA per SM (the registers of kSThreads threads at
// the 128-register cap fill the 64K register file, so no second CTA can contend for TMEM)
template <int M>
void check_sm() {
  if (kSThreads % 128 || kSThreads > 1024) fail("sm threads", M, 0, 0, kSThreads);
  if (kSThreads * 128 != 65536) fail("sm registers do not fill the SM", M, 0, 0, kSThreads * 128);
  if (SmSmem<M>::bytes > kDynMax) fail("sm smem", M, 0, 0, SmSmem<M>::bytes);
  if (SmSmem<M>::oHp < sizeof(float) * 8 * (size_t)kSMaxT) fail("sm r planes", M, 0, 0, SmSmem<M>::oHp);
  if (SmSmem<M>::oQw - SmSmem<M>::oHp < sizeof(float) * (size_t)kSSlots * kSThreads) fail("sm h slots", M, 0, 0, SmSmem<M>::oQw);
  // the Q pass's x blocks sit in the H slots (16 frames x 8 channels per warp)
  if (sizeof(float) * (size_t)kSSlots * kSThreads < sizeof(float) * 2 * 16 * 8 * kSWarps) fail("sm q x blocks", M, 0, 0, 0);
  for (int T = 1; T <= kSMaxT; ++T) {
    const int KF = (T + kSThreads - 1) / kSThreads;
    if (KF > kSSlots || KF * kSThreads < T) fail("sm frame slots", M, 0, T, KF);
    const int warps = kSThreads / 32;
    const int max_col = 128 * ((warps - 1) >> 2) + kSColsPerSlot * (KF - 1) + 15;
    if (max_col >= (int)kSCols || 128 * (warps / 4) > (int)kSCols) fail("sm tmem column", M, 0, T, max_col);
    // the Q pass: warp w takes frames [w per, min((w + 1) per, T)); together they cover [0, T)
    const int per = (T + warps - 1) / warps;
    if (warps * per < T) fail("sm q blocks", M, 0, T, per);
  }
}

template <int M, int N>
void check_frequency_resident() {
  check_em<M, N>();
  check_fca<M, N, false>();
  check_fca<M, N, true>();
  check_mwf<M, N>();
}

template <int M>
void check_all_n() {
  check_frequency_resident<M, 2>();
  check_frequency_resident<M, 3>();
  check_frequency_resident<M, 4>();
  check_frequency_resident<M, 5>();
  check_frequency_resident<M, 6>();
  check_frequency_resident<M, 7>();
  check_frequency_resident<M, 8>();
}

}  // namespace

// tiled filter: the warps' contiguous ranges [gw G / nw, (gw + 1) G / nw) of the G tiles
// cover every tile once, and no two warps' ranges differ by more than one tile
void check_tile_ranges() {
  const int grids[] = {1, 7, 152, 304, 456};
  const long long Gs[] = {1, 3, 255, 1216, 4100, 128125, 256250};
  for (int grid : grids)
    for (long long G : Gs) {
      const long long nw = (long long)grid * kMwfTWarps;
      long long next = 0, lo = G, hi = 0;
      for (long long gw = 0; gw < nw; ++gw) {
        const long long g0 = gw * G / nw, g1 = (gw + 1) * G / nw;
        if (g0 != next || g1 < g0) fail("tile filter tile ranges", grid, 0, (int)G, (int)gw);
        next = g1;
        lo = std::min(lo, g1 - g0);
        hi = std::max(hi, g1 - g0);
      }
      if (next != G || hi - lo > 1) fail("tile filter tile cover", grid, 0, (int)G, (int)(hi - lo));
    }
}

int main() {
  check_tile_ranges();
  check_all_n<2>();
  check_all_n<3>();
  check_all_n<4>();
  check_cluster<2>();
  check_cluster<3>();
  check_cluster<4>();
  check_cluster<5>();
  check_cluster<6>();
  check_cluster<7>();
  check_cluster<8>();
  check_sm<5>();
  check_sm<6>();
  check_sm<7>();
  check_sm<8>();
  if (failures) {
    std::printf("%d violations\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
