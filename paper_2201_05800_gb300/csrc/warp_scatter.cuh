// Warp-level sum of several FP64 accumulators per lane with few FP64 adds.
#pragma once

namespace stdg {

// Warp reduce-scatter of NK accumulators per lane (NK a power of two): at each shuffle
// distance O the lanes split the live accumulators, each half going to the partner lane
// that keeps it, so one step costs NK/2 adds instead of NK; once one accumulator is left
// the remaining distances are a butterfly.  On return a[0] of every lane holds the warp
// sum of accumulator row (all 32/NK lanes of a row hold the same value).
template <int NK, int O>
struct WarpScatter {
  template <int KP>
  static __device__ __forceinline__ void run(double (&a)[KP], int lane, int& row) {
    if constexpr (O > 0) {
      if constexpr (NK > 1) {
        constexpr int H = NK / 2;
        const bool up = (lane & O) != 0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
          const double send = up ? a[i] : a[i + H];
          const double keep = up ? a[i + H] : a[i];
          a[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
        }
        if (up) row += H;
        WarpScatter<H, O / 2>::run(a, lane, row);
      } else {
        a[0] += __shfl_xor_sync(0xffffffffu, a[0], O);
        WarpScatter<1, O / 2>::run(a, lane, row);
      }
    }
  }
};

}  // namespace stdg
