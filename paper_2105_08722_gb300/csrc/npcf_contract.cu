// Contraction of per-primary a^b_lm into the raw multiplets (FP32 CUDA-core path)
// and the FP64 cross-block reduction.
//
// 3PCF (Eq. N=3-coeff with App. B halving):
//   zeta_l(b1,b2) = sum_i u_i (l l 0; 0 0 0) sum_{m=-l..l} a^{b1}_{lm} conj(a^{b2}_{lm})
//                 = sum_i u_i (-1)^l / sqrt(2l+1) [a_{l0} a_{l0} + 2 sum_{m>0} Re(a1 conj a2)].
// Each block owns a chunk of cell-sorted primaries (a range within one catalog); FP32 sums
// over a tile go to the chunk's FP64 partial row, and the reduction adds a catalog's rows
// in chunk order, so results do not depend on scheduling.
#include "npcf_device.h"
#include "npcf_warp.cuh"

namespace npcf {
namespace {

constexpr int kC3Threads = 256;

// A primary's staged a_lm: [b][lm] with an odd stride (in float2), so lanes reading the
// same (b, lm) of different primaries hit different banks.
__host__ __device__ inline int c3_stride(int nr, int nlm) { return (nr * nlm) | 1; }
__host__ __device__ inline size_t c3_su_offset(int nr, int nlm, int T) {
    return ((size_t)T * c3_stride(nr, nlm) * sizeof(float2) + 15) & ~size_t(15);
}
__host__ __device__ inline size_t c3_smem(int nr, int nlm, int T) {
    return c3_su_offset(nr, nlm, T) + (size_t)T * sizeof(float);
}

// Item (l, b1): lane q of the tile adds u_q sum_m f_m Re(a^{b1}_{lm} conj a^{b2}_{lm}) for the
// NB2 shells b2 > b1 (f_0 = 1, f_m = 2), the warp reduces the sums across lanes and adds
// (l l 0; 0 0 0) times them to the outputs (l, b1, b1 + 1 ..), consecutive in the order.
template <int NB2, int T>
__device__ __forceinline__ void c3_item(const int4 item, const float2* __restrict__ X, const float* __restrict__ su,
                                        int nlm, int S, double coef, double* __restrict__ dst, int lane) {
    const int l = item.x, lm0 = item.y, b1 = item.z & 0xff;
    float acc[NB2];
#pragma unroll
    for (int k = 0; k < NB2; ++k) acc[k] = 0.f;
    if (lane < T) {
        const int q = lane;
        const float2* A1 = X + q * S + b1 * nlm + lm0;
        const float u = su[q];
        for (int m = 0; m <= l; ++m) {
            const float2 x1 = A1[m];
            const float f = m == 0 ? u : 2.f * u;
            const float a0 = f * x1.x, a1 = f * x1.y;
#pragma unroll
            for (int k = 0; k < NB2; ++k) {
                const float2 x2 = A1[(k + 1) * nlm + m];
                acc[k] = fmaf(a0, x2.x, fmaf(a1, x2.y, acc[k]));
            }
        }
    }
    using R = warp::TR<NB2>;
    R::run(acc, lane);
#pragma unroll
    for (int i = 0; i < R::F; ++i) {
        const int e = R::origin(i, lane);
        if (e >= 0) dst[item.w + e] += coef * (double)acc[i];
    }
}

// Primaries on the lanes: a block stages the a_lm of T primaries of its chunk (each
// primary's [b][lm] at an odd stride; whole primaries copied by warps, coalesced) and its
// warps take the items (l, b1).
template <int T>
__global__ void __launch_bounds__(kC3Threads) k_contract3(const Contract3Args a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float2* X = reinterpret_cast<float2*>(dsm);
    float* su = reinterpret_cast<float*>(dsm + c3_su_offset(a.nr, a.nlm, T));
    const int chunk = blockIdx.x;
    const int2 C = a.chunks[chunk];   // primaries [C.x, C.y) of one catalog
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rows = a.nr * a.nlm, S = c3_stride(a.nr, a.nlm);
    double* dst = a.partial + (size_t)chunk * a.total + a.out_off;
    for (int i = tid; i < a.nout; i += blockDim.x) dst[i] = 0.0;
    for (int p0 = C.x; p0 < C.y; p0 += T) {
        const int np = min(T, C.y - p0);
        __syncthreads();   // the previous tile is done (and the row is zeroed)
        for (int q = warp; q < T; q += kC3Threads / 32) {
            const float2* src = a.alm + (size_t)(p0 + q) * rows;
            for (int r = lane; r < rows; r += 32) X[q * S + r] = q < np ? src[r] : make_float2(0.f, 0.f);
        }
        if (tid < T) su[tid] = tid < np ? a.wp[p0 + tid] : 0.f;
        __syncthreads();
        // item it always goes to the same warp, so an output is only ever added to by one warp
        for (int it = warp; it < a.nitem; it += kC3Threads / 32) {
            const int4 item = __ldg(&a.items[it]);
            const double coef = (double)__ldg(&a.coef[item.x]);
            switch (item.z >> 16) {
#define NPCF_C3_CASE(K) \
    case K: c3_item<K, T>(item, X, su, a.nlm, S, coef, dst, lane); break;
                NPCF_C3_CASE(1) NPCF_C3_CASE(2) NPCF_C3_CASE(3) NPCF_C3_CASE(4) NPCF_C3_CASE(5)
                NPCF_C3_CASE(6) NPCF_C3_CASE(7) NPCF_C3_CASE(8) NPCF_C3_CASE(9) NPCF_C3_CASE(10)
                NPCF_C3_CASE(11) NPCF_C3_CASE(12) NPCF_C3_CASE(13) NPCF_C3_CASE(14) NPCF_C3_CASE(15)
#undef NPCF_C3_CASE
                default: break;
            }
        }
    }
}

// Catalog blockIdx.y: its chunks' partial rows in order, times the harmonic scale.
__global__ void k_reduce(const double* __restrict__ partial, const int* __restrict__ cbeg, int total, int off,
                         int count, const double* __restrict__ scale, double* __restrict__ zeta) {
    const int e = off + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= off + count) return;
    const int k = blockIdx.y, r0 = cbeg[k], r1 = cbeg[k + 1];
    double s = 0.0;
    for (int c = r0; c < r1; ++c) s += partial[(size_t)c * total + e];
    zeta[(size_t)k * total + e] += s * scale[e];
}

// Sum of weights of catalog blockIdx.y (the blocks along x share its range), added to
// sumw[k] (only the normalisation uses it).
__global__ void k_sumw(const float* __restrict__ w, const long long* __restrict__ off, double* sumw) {
    const int k = blockIdx.y;
    const long long i0 = off[k], i1 = off[k + 1];
    double s = 0.0;
    for (long long i = i0 + blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (long long)gridDim.x * blockDim.x)
        s += w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
        atomicAdd(&sumw[k], t);
    }
}

// Cached harmonics of data primaries (the re-use of the data part across random splits):
// per-primary rows of `row` float2 and `rc` counts moved between cell order and input order.
__global__ void k_alm_to_input(const float2* __restrict__ alm, const uint32_t* __restrict__ cnt,
                               const uint32_t* __restrict__ idx, int n, int row, int rc, float2* __restrict__ alm_in,
                               uint32_t* __restrict__ cnt_in) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * row;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / row), r = (int)(i - (long long)p * row);
        alm_in[(size_t)idx[p] * row + r] = alm[i];
        if (r < rc) cnt_in[(size_t)idx[p] * rc + r] = cnt[(size_t)p * rc + r];
    }
}

__global__ void k_alm_from_input(const float2* __restrict__ alm_in, const uint32_t* __restrict__ cnt_in,
                                 const uint32_t* __restrict__ idx, int n, int row, int rc, float2* __restrict__ alm,
                                 uint32_t* __restrict__ cnt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * row;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i / row), r = (int)(i - (long long)p * row);
        alm[i] = alm_in[(size_t)idx[p] * row + r];
        if (r < rc) cnt[(size_t)p * rc + r] = cnt_in[(size_t)idx[p] * rc + r];
    }
}

__global__ void k_add_counts(unsigned long long* dst, const unsigned long long* src, int n) {
    if (threadIdx.x < n) dst[threadIdx.x] += src[threadIdx.x];
}

__global__ void k_set4(long long* dst, long long a, long long b, long long c, long long d) {
    dst[0] = a;
    dst[1] = b;
    dst[2] = c;
    dst[3] = d;
}

}  // namespace

void launch_alm_to_input(const float2* alm, const uint32_t* cnt, const uint32_t* idx, int n, int row, int rc,
                         float2* alm_in, uint32_t* cnt_in, cudaStream_t s) {
    if (n > 0) k_alm_to_input<<<1024, 256, 0, s>>>(alm, cnt, idx, n, row, rc, alm_in, cnt_in);
}

void launch_alm_from_input(const float2* alm_in, const uint32_t* cnt_in, const uint32_t* idx, int n, int row, int rc,
                           float2* alm, uint32_t* cnt, cudaStream_t s) {
    if (n > 0) k_alm_from_input<<<1024, 256, 0, s>>>(alm_in, cnt_in, idx, n, row, rc, alm, cnt);
}

void launch_add_counts(unsigned long long* dst, const unsigned long long* src, int n, cudaStream_t s) {
    k_add_counts<<<1, 32, 0, s>>>(dst, src, n);
}

void launch_set4(long long* dst, long long a, long long b, long long c, long long d, cudaStream_t s) {
    k_set4<<<1, 1, 0, s>>>(dst, a, b, c, d);
}

void launch_contract3(const Contract3Args& a, cudaStream_t s) {
    if (a.nchunk <= 0 || a.nitem <= 0) return;
    int dev = 0, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // tiles of 32 primaries (a full warp) where they fit, else 16 or 8 (64, two per lane,
    // measured slower: fewer blocks fit on an SM)
    if (c3_smem(a.nr, a.nlm, 32) <= (size_t)optin) {
        cudaFuncSetAttribute(k_contract3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c3_smem(a.nr, a.nlm, 32));
        k_contract3<32><<<a.nchunk, kC3Threads, c3_smem(a.nr, a.nlm, 32), s>>>(a);
    } else if (c3_smem(a.nr, a.nlm, 16) <= (size_t)optin) {
        cudaFuncSetAttribute(k_contract3<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c3_smem(a.nr, a.nlm, 16));
        k_contract3<16><<<a.nchunk, kC3Threads, c3_smem(a.nr, a.nlm, 16), s>>>(a);
    } else {
        cudaFuncSetAttribute(k_contract3<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c3_smem(a.nr, a.nlm, 8));
        k_contract3<8><<<a.nchunk, kC3Threads, c3_smem(a.nr, a.nlm, 8), s>>>(a);
    }
}

void launch_reduce(const double* partial, const int* cbeg, int ncat, int total, int off, int count,
                   const double* scale, double* zeta, cudaStream_t s) {
    if (count <= 0 || ncat <= 0) return;
    k_reduce<<<dim3((count + 255) / 256, ncat), 256, 0, s>>>(partial, cbeg, total, off, count, scale, zeta);
}

void launch_sumw(const float* w, const long long* off, int ncat, double* sumw, cudaStream_t s) {
    if (ncat > 0) k_sumw<<<dim3(32, ncat), 512, 0, s>>>(w, off, sumw);
}

}  // namespace npcf
