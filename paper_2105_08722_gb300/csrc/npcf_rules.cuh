// The neighbour/shell decision shared by every kernel that pairs particles.
#pragma once

namespace npcf {

// IEEE FP32 round-to-nearest, never fused: d = p_j - p_i per axis, minus the periodic
// image shift s of the cell row (0 or +-L, so d - s is exactly the rule's d - L / d + L),
// r2 = (dx*dx + dy*dy) + dz*dz; accepted iff r2 > 0 and e2[0] <= r2 < e2[nr]; the shell
// is the b with e2[b] <= r2 < e2[b+1]. Returns -1 for a rejected pair.
__device__ __forceinline__ int shell_of(const float4 pj, const float4 pi, float sx, float sy,
                                        float sz, const float* e2, int nr) {
    const float dx = __fsub_rn(__fsub_rn(pj.x, pi.x), sx);
    const float dy = __fsub_rn(__fsub_rn(pj.y, pi.y), sy);
    const float dz = __fsub_rn(__fsub_rn(pj.z, pi.z), sz);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (!(r2 > 0.f) || !(r2 >= e2[0]) || !(r2 < e2[nr])) return -1;
    int b = 0;
#pragma unroll
    for (int step = 8; step >= 1; step >>= 1)
        if (b + step < nr && r2 >= e2[b + step]) b += step;
    return b;
}

__device__ __forceinline__ float shift_of(int code, float L) {
    return code == 1 ? L : (code == 2 ? -L : 0.f);
}

}  // namespace npcf
