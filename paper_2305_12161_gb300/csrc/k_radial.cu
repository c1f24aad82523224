// Radially averaged three-dimensional correlation C(r) and structure factor S(k) of one
// lattice (Methods, "Calculating the correlation function": the spin-spin sum for every
// lag vector from FFTs, Eq. (3), then a radial average; Results: S(k,t) is the Fourier
// transform of C).
//
//   1. k_unpack_real: packed spins -> +-1 reals in cuFFT's padded in-place R2C layout
//      (rows of 2(L/2+1) reals).
//   2. cuFFT R2C (library FFT).
//   3. k_power: P(q) = |F(q)|^2 per mode of the half spectrum, summed per radial bin for S
//      (modes with 0 < qx < L/2 stand for their Hermitian partner too), and written back
//      as (P, 0) for the inverse.
//   4. cuFFT C2R: g(k) = sum_q P(q) e^{iqk} = N G(k), G(k) = sum_i s_i s_(i+k).
//   5. k_radial_corr: G(k) = g/N summed per radial bin.  In double precision the FFT error
//      is far below 1/2, so G is rounded to its exact integer and the bin sums are exact
//      (every lag whose g/N lies more than 1/4 from an integer is counted as inexact); in
//      single precision the bin sums are accumulated in double from the rounded-off values.
//   6. k_radial_finish: bin means, C(b) = sum_G / (N n_b), S(b) = sum_P / (N n_b), and the
//      length l at which C first crosses c for r <= L/2.
//
// Bins: components as minimal images, squared length D, bin round(sqrt(D)) computed exactly
// as (isqrt(4D) + 1) / 2.
#include <cufft.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ising {

namespace {

__host__ __device__ __forceinline__ int isqrt_exact(int v)
{
    int s = (int)sqrtf((float)v);  // within one or two of the answer; corrected exactly below
    while (s > 0 && s * s > v) --s;
    while ((s + 1) * (s + 1) <= v) ++s;
    return s;
}

__host__ __device__ __forceinline__ int bin_of(int D) { return (isqrt_exact(4 * D) + 1) >> 1; }

__device__ __forceinline__ int min_image(int j, int L) { return j <= L / 2 ? j : j - L; }

template <typename T>
struct Cx;
template <>
struct Cx<float> {
    using type = cufftComplex;
};
template <>
struct Cx<double> {
    using type = cufftDoubleComplex;
};

constexpr int RAD_THREADS = 256;

}  // namespace

int64_t radial_nbins(int L) { return (int64_t)((isqrt_exact(3 * L * L) + 1) >> 1) + 1; }

// Loops below run over rows (y, z) in a grid-stride loop and over the row's elements with
// the CTA's threads, so no 64-bit division is needed per element.

// 1. A thread takes a pair of sites (x = 2k, 2k+1) of a row: both share compressed index k,
// one on each sublattice.
template <typename T>
__global__ void k_unpack_real(const uint32_t *lat_r, T *buf, Geom g, int64_t P)
{
    const int L = g.L, H = L / 2;
    for (int row = blockIdx.x; row < L * L; row += gridDim.x) {
        const int y = row % L, z = row / L;
        const int q0 = (y + z) & 1;  // sublattice of x = 2k
        const uint32_t *r0 = lat_r + (int64_t)q0 * g.nw + (int64_t)row * g.W;
        const uint32_t *r1 = lat_r + (int64_t)(1 - q0) * g.nw + (int64_t)row * g.W;
        T *dst = buf + (int64_t)row * P;
        for (int k = threadIdx.x; k < H; k += blockDim.x) {
            const int bit = k & 31;
            const uint32_t w0 = __ldg(r0 + (k >> 5)), w1 = __ldg(r1 + (k >> 5));
            dst[2 * k] = ((w0 >> bit) & 1u) ? T(1) : T(-1);
            dst[2 * k + 1] = ((w1 >> bit) & 1u) ? T(1) : T(-1);
        }
    }
}

// Per-CTA bins in shared memory, flushed to the global sums at the end.
template <typename T>
__global__ void __launch_bounds__(RAD_THREADS) k_power(typename Cx<T>::type *F, int L, int nb, double *sumS)
{
    extern __shared__ double hs[];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hs[i] = 0.0;
    __syncthreads();
    const int H1 = L / 2 + 1;
    for (int row = blockIdx.x; row < L * L; row += gridDim.x) {
        const int ny = min_image(row % L, L), nz = min_image(row / L, L);
        const int dyz = ny * ny + nz * nz;
        typename Cx<T>::type *Fr = F + (int64_t)row * H1;
        for (int nx = threadIdx.x; nx < H1; nx += blockDim.x) {
            const typename Cx<T>::type f = Fr[nx];
            const double p = (double)f.x * (double)f.x + (double)f.y * (double)f.y;
            const double w = (nx == 0 || nx == L / 2) ? 1.0 : 2.0;
            atomicAdd(&hs[bin_of(nx * nx + dyz)], w * p);
            typename Cx<T>::type o;
            o.x = (T)p;
            o.y = T(0);
            Fr[nx] = o;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (hs[i] != 0.0) atomicAdd(&sumS[i], hs[i]);
}

// EXACT: round g/N to the integer G(k) and sum integers (double precision transforms).
template <typename T, bool EXACT>
__global__ void __launch_bounds__(RAD_THREADS) k_radial_corr(const T *g, int L, int64_t P, int nb, double invN,
                                                             long long *sumG, double *sumC,
                                                             unsigned long long *count, unsigned long long *inexact)
{
    extern __shared__ long long hsm[];
    long long *hG = hsm;                                              // EXACT: integer sums
    double *hC = reinterpret_cast<double *>(hsm);                     // otherwise: real sums
    unsigned long long *hn = reinterpret_cast<unsigned long long *>(hsm + nb);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        hG[i] = 0;
        hn[i] = 0ull;
    }
    __syncthreads();
    unsigned long long bad = 0ull;
    for (int row = blockIdx.x; row < L * L; row += gridDim.x) {
        const int dy = min_image(row % L, L), dz = min_image(row / L, L);
        const int dyz = dy * dy + dz * dz;
        const T *gr = g + (int64_t)row * P;
        for (int x = threadIdx.x; x < L; x += blockDim.x) {
            const int dx = min_image(x, L);
            const int b = bin_of(dx * dx + dyz);
            const double v = (double)gr[x] * invN;
            if (EXACT) {
                const double r = rint(v);
                if (fabs(v - r) > 0.25) ++bad;
                atomicAdd(reinterpret_cast<unsigned long long *>(&hG[b]), (unsigned long long)(long long)r);
            } else {
                atomicAdd(&hC[b], v);
            }
            atomicAdd(&hn[b], 1ull);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        if (hn[i] == 0ull) continue;
        if (EXACT)
            atomicAdd(reinterpret_cast<unsigned long long *>(&sumG[i]), (unsigned long long)hG[i]);
        else
            atomicAdd(&sumC[i], hC[i]);
        atomicAdd(&count[i], hn[i]);
    }
    if (EXACT && bad) atomicAdd(inexact, bad);
}

// out = [C(0..nb-1), S(0..nb-1), l]; cnt = [n_b (nb), inexact lags].
__global__ void k_radial_finish(int L, int nb, int exact, double c, const long long *sumG, const double *sumC,
                                const double *sumS, const unsigned long long *count,
                                const unsigned long long *inexact, double *out, int64_t *cnt)
{
    const double N = (double)L * (double)L * (double)L;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double n = (double)count[b];
        const double denom = __dmul_rn(N, n);
        const double num = exact ? (double)sumG[b] : sumC[b];  // the bin's sum of G(k)
        out[b] = count[b] ? __ddiv_rn(num, denom) : 0.0;
        out[nb + b] = count[b] ? __ddiv_rn(sumS[b], denom) : 0.0;
        cnt[b] = (int64_t)count[b];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ell = __longlong_as_double(0x7ff8000000000000ll);  // NaN: no crossing
        for (int r = 0; r < L / 2; ++r) {
            const double c0 = out[r], c1 = out[r + 1];
            if (c0 >= c && c > c1) {
                ell = __dadd_rn((double)r, __ddiv_rn(__dsub_rn(c0, c), __dsub_rn(c0, c1)));
                break;
            }
        }
        out[2 * nb] = ell;
        cnt[nb] = exact ? (int64_t)*inexact : -1;
    }
}

// ---------------------------------------------------------------------------------
struct RadialPlans {
    int L = 0;
    bool made[2] = {false, false};
    cufftHandle fwd[2] = {0, 0}, inv[2] = {0, 0};
    size_t work[2] = {0, 0};
};

RadialPlans *radial_plans_create() { return new (std::nothrow) RadialPlans(); }

void radial_plans_destroy(RadialPlans *p)
{
    if (!p) return;
    for (int i = 0; i < 2; ++i)
        if (p->made[i]) {
            cufftDestroy(p->fwd[i]);
            cufftDestroy(p->inv[i]);
        }
    delete p;
}

static int make_plans(RadialPlans *p, int L, int prec)
{
    if (p->made[prec]) return CUFFT_SUCCESS;
    long long n[3] = {L, L, L};
    size_t w1 = 0, w2 = 0;
    cufftResult r;
    if ((r = cufftCreate(&p->fwd[prec])) != CUFFT_SUCCESS) return r;
    if ((r = cufftCreate(&p->inv[prec])) != CUFFT_SUCCESS) {
        cufftDestroy(p->fwd[prec]);
        return r;
    }
    cufftSetAutoAllocation(p->fwd[prec], 0);
    cufftSetAutoAllocation(p->inv[prec], 0);
    r = cufftMakePlanMany64(p->fwd[prec], 3, n, nullptr, 1, 0, nullptr, 1, 0, prec ? CUFFT_D2Z : CUFFT_R2C, 1, &w1);
    if (r == CUFFT_SUCCESS)
        r = cufftMakePlanMany64(p->inv[prec], 3, n, nullptr, 1, 0, nullptr, 1, 0, prec ? CUFFT_Z2D : CUFFT_C2R, 1,
                                &w2);
    if (r != CUFFT_SUCCESS) {
        cufftDestroy(p->fwd[prec]);
        cufftDestroy(p->inv[prec]);
        return r;
    }
    p->L = L;
    p->work[prec] = std::max(w1, w2);
    p->made[prec] = true;
    return CUFFT_SUCCESS;
}

size_t radial_scratch_bytes(int L, int prec)
{
    const size_t elem = prec ? sizeof(double) : sizeof(float);
    return (size_t)L * (size_t)L * (size_t)(L / 2 + 1) * 2 * elem;
}

template <typename T>
static cudaError_t run_radial(RadialPlans *p, const uint32_t *lat_r, int L, double c, double *out, int64_t *cnt,
                              cudaStream_t s, int64_t *launches, int *cufft_status)
{
    constexpr int prec = sizeof(T) == 8 ? 1 : 0;
    const Geom g = make_geom(L);
    const int nb = (int)radial_nbins(L);
    const int64_t P = 2 * (int64_t)(L / 2 + 1);
    int cs = make_plans(p, L, prec);
    if (cs != CUFFT_SUCCESS) {
        *cufft_status = cs;
        return cudaErrorUnknown;
    }
    const size_t data_bytes = radial_scratch_bytes(L, prec);
    const size_t acc_bytes = (size_t)nb * (3 * sizeof(double) + sizeof(unsigned long long)) + 64;
    char *buf = nullptr, *work = nullptr, *acc = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&buf, data_bytes, s);
    if (e != cudaSuccess) return e;
    if (p->work[prec] && (e = cudaMallocAsync((void **)&work, p->work[prec], s)) != cudaSuccess) {
        cudaFreeAsync(buf, s);
        return e;
    }
    if ((e = cudaMallocAsync((void **)&acc, acc_bytes, s)) != cudaSuccess) {
        cudaFreeAsync(buf, s);
        if (work) cudaFreeAsync(work, s);
        return e;
    }
    auto cleanup = [&](cudaError_t err) {
        cudaFreeAsync(acc, s);
        if (work) cudaFreeAsync(work, s);
        cudaFreeAsync(buf, s);
        return err;
    };
    long long *sumG = reinterpret_cast<long long *>(acc);
    double *sumC = reinterpret_cast<double *>(acc);  // same storage: one of the two is used
    double *sumS = reinterpret_cast<double *>(acc) + nb;
    unsigned long long *count = reinterpret_cast<unsigned long long *>(acc) + 2 * nb;
    unsigned long long *inexact = count + nb;
    if ((e = cudaMemsetAsync(acc, 0, acc_bytes, s)) != cudaSuccess) return cleanup(e);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms * 4);

    k_unpack_real<T><<<grid, RAD_THREADS, 0, s>>>(lat_r, reinterpret_cast<T *>(buf), g, P);
    cufftHandle f = p->fwd[prec], iv = p->inv[prec];
    if ((cs = cufftSetStream(f, s)) != CUFFT_SUCCESS || (cs = cufftSetStream(iv, s)) != CUFFT_SUCCESS ||
        (cs = cufftSetWorkArea(f, work)) != CUFFT_SUCCESS || (cs = cufftSetWorkArea(iv, work)) != CUFFT_SUCCESS) {
        *cufft_status = cs;
        return cleanup(cudaErrorUnknown);
    }
    using C = typename Cx<T>::type;
    if (prec)
        cs = cufftExecD2Z(f, reinterpret_cast<cufftDoubleReal *>(buf), reinterpret_cast<cufftDoubleComplex *>(buf));
    else
        cs = cufftExecR2C(f, reinterpret_cast<cufftReal *>(buf), reinterpret_cast<cufftComplex *>(buf));
    if (cs != CUFFT_SUCCESS) {
        *cufft_status = cs;
        return cleanup(cudaErrorUnknown);
    }
    const size_t smem_p = (size_t)nb * sizeof(double);
    if ((e = cudaFuncSetAttribute(k_power<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p)) != cudaSuccess)
        return cleanup(e);
    k_power<T><<<grid, RAD_THREADS, smem_p, s>>>(reinterpret_cast<C *>(buf), L, nb, sumS);
    if (prec)
        cs = cufftExecZ2D(iv, reinterpret_cast<cufftDoubleComplex *>(buf), reinterpret_cast<cufftDoubleReal *>(buf));
    else
        cs = cufftExecC2R(iv, reinterpret_cast<cufftComplex *>(buf), reinterpret_cast<cufftReal *>(buf));
    if (cs != CUFFT_SUCCESS) {
        *cufft_status = cs;
        return cleanup(cudaErrorUnknown);
    }
    const size_t smem_c = (size_t)nb * 2 * sizeof(long long);
    const double invN = 1.0 / ((double)L * (double)L * (double)L);  // exact: N is a power of two
    if (prec) {
        if ((e = cudaFuncSetAttribute(k_radial_corr<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_c)) != cudaSuccess)
            return cleanup(e);
        k_radial_corr<T, true><<<grid, RAD_THREADS, smem_c, s>>>(reinterpret_cast<const T *>(buf), L, P, nb, invN,
                                                                  sumG, sumC, count, inexact);
    } else {
        if ((e = cudaFuncSetAttribute(k_radial_corr<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_c)) != cudaSuccess)
            return cleanup(e);
        k_radial_corr<T, false><<<grid, RAD_THREADS, smem_c, s>>>(reinterpret_cast<const T *>(buf), L, P, nb, invN,
                                                                   sumG, sumC, count, inexact);
    }
    k_radial_finish<<<1, 256, 0, s>>>(L, nb, prec, c, sumG, sumC, sumS, count, inexact, out, cnt);
    if (launches) *launches += 4;  // own kernels; the two cuFFT executions are library launches
    return cleanup(cudaGetLastError());
}

cudaError_t launch_radial(RadialPlans *p, const uint32_t *lat_r, int L, int precision, double c, double *out,
                          int64_t *cnt, cudaStream_t s, int64_t *launches, int *cufft_status)
{
    *cufft_status = CUFFT_SUCCESS;
    if (precision)
        return run_radial<double>(p, lat_r, L, c, out, cnt, s, launches, cufft_status);
    return run_radial<float>(p, lat_r, L, c, out, cnt, s, launches, cufft_status);
}

}  // namespace ising
