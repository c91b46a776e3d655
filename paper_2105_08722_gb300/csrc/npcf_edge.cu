// Edge correction of the raw multiplets (a7), FP64 on the GPU.
//
// Eq. (edge-corrected-NPCF) with the basis-function product of Eq. (basis-function-product):
// for each bin tuple B the edge-corrected zeta_L(B) solve
//   sum_L zeta_L(B) M_{L L''}(B) = N_{L''}(B) / R_0(B),
//   M_{L L''}(B) = sum_{L'} f_{L'}(B) E(L'') G^{L L' L''},   f_{L'} = R_{L'}(B) / R_0(B),
// where N are the raw multiplets of the data-minus-randoms run, R those of the randoms-only
// run and G the generalized Gaunt integrals of App. A. Only parity-even multiplets enter
// (E(L'') = +1). One block per B builds M from a sparse table of G (rows grouped by the
// matrix entry they feed, so every entry is one thread's ordered sum) and solves the
// system by Gaussian elimination with partial pivoting in shared memory.
#include "npcf_device.h"

namespace npcf {
namespace {

__global__ void k_edge_solve(const EdgeArgs a) {
    extern __shared__ __align__(16) double esm[];
    const int nl = a.nl, nb = a.nb, B = blockIdx.x;
    double* M = esm;              // [nl][nl], row = equation L'', column = unknown L
    double* x = M + nl * nl;      // right-hand side, then the solution
    double* f = x + nl;           // R_{L'} / R_0
    __shared__ int piv, singular;
    __shared__ double pval;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const double R0 = a.rraw[B];   // multiplet 0 is L = (0, ..., 0)
    if (tid == 0) singular = (R0 == 0.0 || !isfinite(R0)) ? 1 : 0;
    for (int i = tid; i < nl; i += blockDim.x) {
        f[i] = a.rraw[(size_t)i * nb + B] / R0;
        x[i] = a.nraw[(size_t)i * nb + B] / R0;
    }
    __syncthreads();
    for (int e = tid; e < nl * nl; e += blockDim.x) {
        double s = 0.0;
        for (int k = a.tptr[e]; k < a.tptr[e + 1]; ++k) s += f[a.tlp[k]] * a.tg[k];
        M[e] = s;
    }
    __syncthreads();

    for (int k = 0; k < nl && !singular; ++k) {
        if (warp == 0) {
            // pivot: largest |M[r][k]| for r >= k (smallest r among equals)
            double best = -1.0;
            int br = k;
            for (int r = k + lane; r < nl; r += 32) {
                const double v = fabs(M[r * nl + k]);
                if (v > best) { best = v; br = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int orow = __shfl_xor_sync(0xffffffffu, br, o);
                if (ov > best || (ov == best && orow < br)) { best = ov; br = orow; }
            }
            if (lane == 0) {
                piv = br;
                pval = best;
                if (!(best > 0.0)) singular = 1;
            }
        }
        __syncthreads();
        if (singular) break;
        const int p = piv;
        if (p != k) {
            for (int j = k + tid; j < nl; j += blockDim.x) {
                const double t = M[k * nl + j];
                M[k * nl + j] = M[p * nl + j];
                M[p * nl + j] = t;
            }
            if (tid == 0) {
                const double t = x[k];
                x[k] = x[p];
                x[p] = t;
            }
        }
        __syncthreads();
        // rows below: subtract (M[r][k] / M[k][k]) times row k; column k itself is left as
        // it is (back substitution reads only j > r), column nl stands for x
        const int w = nl - k;   // columns k+1 .. nl
        const double inv = 1.0 / M[k * nl + k];
        for (int e = tid; e < (nl - k - 1) * w; e += blockDim.x) {
            const int r = k + 1 + e / w, j = k + 1 + e % w;
            const double fac = M[r * nl + k] * inv;
            if (j < nl) M[r * nl + j] -= fac * M[k * nl + j];
            else x[r] -= fac * x[k];
        }
        __syncthreads();
    }
    // back substitution, one row at a time with a block-wide dot product
    __shared__ double part[32];
    for (int r = nl - 1; r >= 0 && !singular; --r) {
        double s = 0.0;
        for (int j = r + 1 + tid; j < nl; j += blockDim.x) s += M[r * nl + j] * x[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
            x[r] = (x[r] - t) / M[r * nl + r];
        }
        __syncthreads();
    }
    if (singular) {
        if (tid == 0) atomicOr(a.err, 4);
        for (int i = tid; i < nl; i += blockDim.x) a.out[(size_t)i * nb + B] = nan("");
        return;
    }
    for (int i = tid; i < nl; i += blockDim.x) a.out[(size_t)i * nb + B] = x[i];
}

}  // namespace

size_t edge_smem_bytes(int nl) { return ((size_t)nl * nl + 2 * (size_t)nl) * sizeof(double); }

void launch_edge_solve(const EdgeArgs& a, cudaStream_t s) {
    const size_t smem = edge_smem_bytes(a.nl);
    cudaFuncSetAttribute(k_edge_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_edge_solve<<<a.nb, 256, smem, s>>>(a);
}

}  // namespace npcf
