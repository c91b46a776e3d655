// Warp-level helpers shared by the kernels.
#pragma once

namespace npcf {
namespace warp {

constexpr unsigned kFullMask = 0xffffffffu;

// One halving step of the warp transpose-reduction: values [0, C) pair with
// [H, 2H); lanes with bit O set keep the upper half.
template <int C, int O>
__device__ __forceinline__ void tr_step(float* v, int lane) {
    constexpr int H = (C + 1) / 2;
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float lo = v[i];
        float hi = (i + H < C) ? v[i + H] : 0.f;
        float send = up ? lo : hi;
        float keep = up ? hi : lo;
        v[i] = keep + __shfl_xor_sync(kFullMask, send, O);
    }
}

// Transpose-reduction of V per-lane values over the 32 lanes of a warp: afterwards
// lane l holds F sums, final slot i being the sum of original value origin(i, l).
template <int V>
struct TR {
    static constexpr int C0 = V, C1 = (C0 + 1) / 2, C2 = (C1 + 1) / 2, C3 = (C2 + 1) / 2,
                         C4 = (C3 + 1) / 2, C5 = (C4 + 1) / 2;
    static constexpr int F = C5;   // values left per lane
    __device__ static void run(float* v, int lane) {
        tr_step<C0, 16>(v, lane);
        tr_step<C1, 8>(v, lane);
        tr_step<C2, 4>(v, lane);
        tr_step<C3, 2>(v, lane);
        tr_step<C4, 1>(v, lane);
    }
    // original index of final slot i on this lane, or -1 for a padding slot
    __device__ static int origin(int i, int lane) {
        const int Cs[5] = {C0, C1, C2, C3, C4};
        const int Os[5] = {16, 8, 4, 2, 1};
        int idx = i;
        for (int st = 4; st >= 0; --st) {
            int H = (Cs[st] + 1) / 2;
            if (lane & Os[st]) idx += H;
            if (idx >= Cs[st]) return -1;
        }
        return idx;
    }
};

}  // namespace warp
}  // namespace npcf
