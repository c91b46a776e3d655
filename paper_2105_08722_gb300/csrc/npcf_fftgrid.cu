// Harmonic coefficients of a density field on a periodic grid by FFT (Sec. 3.2.2,
// Eq. alm-binned-def-fft): for every cell s of an n^3 mesh (cell side h = L / n, cells x
// fastest) and every shell b,
//   a^b_lm(s) = sum_t delta(t) Y_lm(unit(r_t - r_s)) Theta^b(|r_t - r_s|),
// the discrete estimator's a_lm with the cells as particles of weight delta at their
// centres (without 1/v_b: raw sums). The shell of a cell offset is decided by the same
// FP32 rule as the particle path, on the offset's separation vector Delta h (periodic: the
// minimum image, Delta in [-n/2, n/2)). Taken on the separation r_t - r_s (the reading of
// Eq. binned-discrete-alm used throughout), the field is a circular correlation; with the
// kernel K(u) = Y_lm(unit(-u h)) Theta^b(|u h|) it is the circular convolution K * delta,
// i.e. the inverse FFT of FFT(K) FFT(delta) divided by n^3 (Eq. alm-binned-def-fft on the
// mirrored kernel: a factor (-1)^l from the paper's form). The kernel spectra of every (b, l,
// m >= 0) depend only on the mesh and are kept between calls. Transforms are FP32 (cuFFT
// C2C; the kernel values are computed in FP64): their rounding, about 1e-6 of the RMS of the
// a_lm on a 64^3 log-normal field, is far below the FP32 contraction's error bar, and FP64
// transforms ran at the GPU's much lower FP64 rate. The a_lm are stored as FP32 reduced
// harmonics a_lm / sqrt((2l+1)/(4 pi)), the layout the contraction kernels read, with the
// cells as primaries.
#include "npcf_device.h"

#include <cufft.h>

#include <cmath>
#include <cstdio>

namespace npcf {

struct GridFFT {
    int n = 0, nr = 0, lmax = -1;
    float h = 0.f;
    float e2[kMaxNr + 1] = {};
    float2* spec = nullptr;     // [nr][nlm][n^3] kernel spectra
    float2* df = nullptr;       // [n^3] spectrum of delta
    float2* work = nullptr;     // [nlm][n^3]
    cufftHandle one = 0, many = 0;
    bool plans = false;
    void release() {
        if (plans) {
            cufftDestroy(one);
            cufftDestroy(many);
            plans = false;
        }
        if (spec) cudaFree(spec);
        if (df) cudaFree(df);
        if (work) cudaFree(work);
        spec = df = work = nullptr;
        n = 0;
    }
    ~GridFFT() { release(); }
};

GridFFT* gridfft_create() { return new GridFFT(); }
void gridfft_destroy(GridFFT* g) { delete g; }

namespace {

__host__ __device__ constexpr int nlm_of(int L) { return (L + 1) * (L + 2) / 2; }

// Kernel of shell b on the mesh, for every (l, m >= 0): K(u) = Y~_lm(unit(-u h)) where the
// FP32 rule puts the offset in shell b, else 0; Y~_lm = sqrt((l-m)!/(l+m)!) P_l^m(z) e^{i m phi}
// (Condon-Shortley phase), written as (x + i y)^m times a polynomial in z.
__global__ void k_mesh_kernel(float2* __restrict__ out, int n, float h, const GridFFTArgs a, int b) {
    const long long cells = (long long)n * n * n;
    const int nlm = nlm_of(a.lmax);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
         c += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(c % n), iy = (int)((c / n) % n), iz = (int)(c / ((long long)n * n));
        const int ux = ix < (n + 1) / 2 ? ix : ix - n, uy = iy < (n + 1) / 2 ? iy : iy - n,
                  uz = iz < (n + 1) / 2 ? iz : iz - n;
        // separation of the mirrored offset, exactly as the rule forms it from cell centres
        const float dx = __fmul_rn((float)(-ux), h), dy = __fmul_rn((float)(-uy), h), dz = __fmul_rn((float)(-uz), h);
        const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        int sb = -1;
        if (r2 > 0.f && r2 >= a.e2[0] && r2 < a.e2[a.nr]) {
            sb = 0;
            while (sb + 1 < a.nr && r2 >= a.e2[sb + 1]) ++sb;
        }
        if (sb != b) {
            for (int q = 0; q < nlm; ++q) out[(size_t)q * cells + c] = make_float2(0.f, 0.f);
            continue;
        }
        const double r = sqrt((double)r2);
        const double x = dx / r, y = dy / r, z = dz / r;
        double cr = 1.0, ci = 0.0;          // (x + i y)^m
        double qmm = 1.0;                   // (-1)^m (2m-1)!!
        double fac = 1.0;                   // (l-m)!/(l+m)! at l = m: 1/(2m)!
        for (int m = 0; m <= a.lmax; ++m) {
            if (m > 0) {
                const double t = cr * x - ci * y;
                ci = cr * y + ci * x;
                cr = t;
                qmm *= -(2.0 * m - 1.0);
                fac /= (2.0 * m) * (2.0 * m - 1.0);
            }
            double q0 = qmm, q1 = 0.0, f = fac;
            for (int l = m; l <= a.lmax; ++l) {
                double ql;
                if (l == m) {
                    ql = q0;
                } else if (l == m + 1) {
                    q1 = z * (2.0 * m + 1.0) * q0;
                    ql = q1;
                } else {
                    ql = ((2.0 * l - 1.0) * z * q1 - (l + m - 1.0) * q0) / (double)(l - m);
                    q0 = q1;
                    q1 = ql;
                }
                if (l > m) f *= (double)(l - m) / (double)(l + m);
                const double s = sqrt(f) * ql;
                out[(size_t)(l * (l + 1) / 2 + m) * cells + c] = make_float2((float)(s * cr), (float)(s * ci));
            }
        }
    }
}

__global__ void k_delta_complex(float2* __restrict__ out, const float* __restrict__ delta, long long cells) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
         c += (long long)gridDim.x * blockDim.x)
        out[c] = make_float2(delta[c], 0.f);
}

// work[q][c] = spec[q][c] * df[c] for every harmonic q
__global__ void k_spectral_mul(float2* __restrict__ work, const float2* __restrict__ spec,
                               const float2* __restrict__ df, long long cells, int nlm) {
    const long long tot = cells * nlm;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 k = spec[i], d = df[i % cells];
        work[i] = make_float2(k.x * d.x - k.y * d.y, k.x * d.y + k.y * d.x);
    }
}

// alm[c][b][q] = work[q][c] / n^3
__global__ void k_store_alm(const float2* __restrict__ work, float2* __restrict__ alm, long long cells, int nlm,
                            int nr, int b, float scale) {
    const long long tot = cells * nlm;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = i / nlm;
        const int q = (int)(i - c * nlm);
        const float2 v = work[(size_t)q * cells + c];
        alm[((size_t)c * nr + b) * nlm + q] = make_float2(v.x * scale, v.y * scale);
    }
}

__global__ void k_copy_weights(float* __restrict__ wp, const float* __restrict__ delta, long long cells) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
         c += (long long)gridDim.x * blockDim.x)
        wp[c] = delta[c];
}

int blocks_for(long long work) {
    const long long b = (work + 255) / 256;
    return (int)(b < 8192 ? (b > 0 ? b : 1) : 8192);
}

}  // namespace

int gridfft_alm(GridFFT* G, const float* delta, int n, float box, const GridFFTArgs& a, float2* alm, float* wp,
                cudaStream_t s, char* err, size_t errlen) {
    const long long cells = (long long)n * n * n;
    const int nlm = nlm_of(a.lmax);
    const float h = (float)((double)box / n);
    auto cuda_fail = [&](const char* what, cudaError_t e) {
        snprintf(err, errlen, "%s: %s", what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? 2 : 3;
    };
    auto fft_fail = [&](const char* what, cufftResult r) {
        snprintf(err, errlen, "%s: cuFFT error %d", what, (int)r);
        return r == CUFFT_ALLOC_FAILED ? 2 : 3;
    };
    bool same = G->n == n && G->nr == a.nr && G->lmax == a.lmax && G->h == h;
    for (int i = 0; same && i <= a.nr; ++i) same = G->e2[i] == a.e2[i];
    if (!same) {
        G->release();
        cudaError_t e;
        if ((e = cudaMalloc(&G->spec, sizeof(float2) * (size_t)a.nr * nlm * cells)) != cudaSuccess)
            return cuda_fail("kernel spectra", e);
        if ((e = cudaMalloc(&G->df, sizeof(float2) * (size_t)cells)) != cudaSuccess) return cuda_fail("delta spectrum", e);
        if ((e = cudaMalloc(&G->work, sizeof(float2) * (size_t)nlm * cells)) != cudaSuccess)
            return cuda_fail("harmonic fields", e);
        cufftResult r;
        if ((r = cufftPlan3d(&G->one, n, n, n, CUFFT_C2C)) != CUFFT_SUCCESS) return fft_fail("plan", r);
        int dims[3] = {n, n, n};
        if ((r = cufftPlanMany(&G->many, 3, dims, nullptr, 1, (int)cells, nullptr, 1, (int)cells, CUFFT_C2C, nlm)) !=
            CUFFT_SUCCESS) {
            cufftDestroy(G->one);
            return fft_fail("batched plan", r);
        }
        G->plans = true;
        // cuFFT's x is its last (fastest) dimension: dims (n, n, n) over [z][y][x] storage
        if ((r = cufftSetStream(G->many, s)) != CUFFT_SUCCESS) return fft_fail("stream", r);
        for (int b = 0; b < a.nr; ++b) {
            float2* sb = G->spec + (size_t)b * nlm * cells;
            k_mesh_kernel<<<blocks_for(cells), 256, 0, s>>>(sb, n, h, a, b);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("mesh kernel", e);
            if ((r = cufftExecC2C(G->many, (cufftComplex*)sb, (cufftComplex*)sb, CUFFT_FORWARD)) !=
                CUFFT_SUCCESS)
                return fft_fail("kernel transform", r);
        }
        G->n = n;
        G->nr = a.nr;
        G->lmax = a.lmax;
        G->h = h;
        for (int i = 0; i <= a.nr; ++i) G->e2[i] = a.e2[i];
    }
    cufftResult r;
    if ((r = cufftSetStream(G->one, s)) != CUFFT_SUCCESS || (r = cufftSetStream(G->many, s)) != CUFFT_SUCCESS)
        return fft_fail("stream", r);
    k_delta_complex<<<blocks_for(cells), 256, 0, s>>>(G->df, delta, cells);
    if ((r = cufftExecC2C(G->one, (cufftComplex*)G->df, (cufftComplex*)G->df, CUFFT_FORWARD)) !=
        CUFFT_SUCCESS)
        return fft_fail("delta transform", r);
    for (int b = 0; b < a.nr; ++b) {
        k_spectral_mul<<<blocks_for(cells * nlm), 256, 0, s>>>(G->work, G->spec + (size_t)b * nlm * cells, G->df,
                                                              cells, nlm);
        if ((r = cufftExecC2C(G->many, (cufftComplex*)G->work, (cufftComplex*)G->work, CUFFT_INVERSE)) !=
            CUFFT_SUCCESS)
            return fft_fail("inverse transform", r);
        k_store_alm<<<blocks_for(cells * nlm), 256, 0, s>>>(G->work, alm, cells, nlm, a.nr, b, (float)(1.0 / (double)cells));
    }
    k_copy_weights<<<blocks_for(cells), 256, 0, s>>>(wp, delta, cells);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("grid kernels", e);
    return 0;
}

}  // namespace npcf
