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
//   5. k_radial_corr: G(k) = g/N rounded to the nearest integer and summed per radial bin in
//      int64.  G(k) is an integer; when the FFT error stays below 1/2 (always in double
//      precision, at small L in single) the rounding recovers it exactly and C is exact.  A
//      lag whose g/N lies more than 1/4 from an integer is counted as inexact.
//   6. k_radial_finish: bin means, C(b) = sum_G / (N n_b), S(b) = sum_P / (N n_b), and the
//      length l at which C first crosses c for r <= L/2.
//
// Binning: the lanes of a warp take consecutive elements of a row, whose bins form runs; a
// segmented warp scan sums each run and its last lane adds the sum to the CTA's bins in
// shared memory with one atomic, and the CTA's bins go to the global sums at the end.  The
// number of vectors per bin does not depend on the state and is counted once per context.
// The transform buffer and cuFFT's work area stay allocated in the context between calls.
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

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

constexpr int RAD_THREADS = 256;

}  // namespace

int64_t radial_nbins(int L) { return (int64_t)((isqrt_exact(3 * L * L) + 1) >> 1) + 1; }

// Loops below run over rows (y, z) in a grid-stride loop and over the row's elements with
// the CTA's warps, lane = consecutive element, so no 64-bit division is needed per element.

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
            typename Pair<T>::type v;  // one aligned store of the two sites (rows of even length)
            v.x = ((w0 >> bit) & 1u) ? T(1) : T(-1);
            v.y = ((w1 >> bit) & 1u) ? T(1) : T(-1);
            *reinterpret_cast<typename Pair<T>::type *>(dst + 2 * k) = v;
        }
    }
}

// The 32 lanes hold (bin b, value v) of consecutive elements (b < 0: no element).  Runs of
// equal b are summed by a segmented inclusive scan in type V; each run's last lane adds its
// sum to hist[b] (type H).
template <typename V, typename H>
__device__ __forceinline__ void run_add(int b, V v, H *hist)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int bp = __shfl_up_sync(FULL, b, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0 || bp != b);
    const int seg = __popc(heads & (FULL >> (31 - lane)));  // run number of this lane
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const V vo = __shfl_up_sync(FULL, v, d);
        const int so = __shfl_up_sync(FULL, seg, d);
        if (lane >= d && so == seg) v += vo;
    }
    const int bn = __shfl_down_sync(FULL, b, 1);
    if ((lane == 31 || bn != b) && b >= 0) atomicAdd(&hist[b], (H)v);
}

template <typename V>
__device__ __forceinline__ void zero_bins(V *h, int nb)
{
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = V(0);
    __syncthreads();
}

template <typename V>
__device__ __forceinline__ void flush_bins(const V *h, V *global, int nb)
{
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (h[i] != V(0)) atomicAdd(&global[i], h[i]);
}

// 3. |F|^2 per mode of the half spectrum; S sums per bin; (P, 0) written back.
template <typename T>
__global__ void __launch_bounds__(RAD_THREADS) k_power(typename Cx<T>::type *F, int L, int nb, double *sumS)
{
    extern __shared__ double hs[];
    zero_bins(hs, nb);
    const int H1 = L / 2 + 1;
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x; row < L * L; row += gridDim.x) {
        const int ny = min_image(row % L, L), nz = min_image(row / L, L);
        const int dyz = ny * ny + nz * nz;
        typename Cx<T>::type *Fr = F + (int64_t)row * H1;
        for (int x0 = threadIdx.x & ~31; x0 < H1; x0 += blockDim.x) {
            const int nx = x0 + lane;
            int b = -1;
            T wp = T(0);  // single precision stays in fp32 up to the per-run double add
            if (nx < H1) {
                const typename Cx<T>::type f = Fr[nx];
                const T p = f.x * f.x + f.y * f.y;
                wp = (nx == 0 || nx == L / 2) ? p : T(2) * p;  // 0 < nx < L/2: also the partner -q
                b = bin_of(nx * nx + dyz);
                typename Cx<T>::type o;
                o.x = p;
                o.y = T(0);
                Fr[nx] = o;
            }
            run_add<T, double>(b, wp, hs);
        }
    }
    flush_bins(hs, sumS, nb);
}

// 5. G(k) = rint(g/N) per lag, summed per bin in int64.
template <typename T>
__global__ void __launch_bounds__(RAD_THREADS) k_radial_corr(const T *g, int L, int64_t P, int nb, double invN,
                                                             unsigned long long *sumG, unsigned long long *inexact)
{
    extern __shared__ unsigned long long hg[];
    zero_bins(hg, nb);
    const int lane = threadIdx.x & 31;
    unsigned long long bad = 0ull;
    for (int row = blockIdx.x; row < L * L; row += gridDim.x) {
        const int dy = min_image(row % L, L), dz = min_image(row / L, L);
        const int dyz = dy * dy + dz * dz;
        const T *gr = g + (int64_t)row * P;
        for (int x0 = threadIdx.x & ~31; x0 < L; x0 += blockDim.x) {
            const int x = x0 + lane;
            int b = -1;
            unsigned long long G = 0ull;
            if (x < L) {
                const int dx = min_image(x, L);
                b = bin_of(dx * dx + dyz);
                // invN is a power of two, so the scaling is exact in either precision
                const T v = gr[x] * (T)invN;
                const T r = rint(v);
                if (fabs(v - r) > T(0.25)) ++bad;
                // two's complement: the unsigned sums wrap to the signed result
                G = (fabs(r) < T(2147483520)) ? (unsigned long long)(long long)(int)r
                                               : (unsigned long long)(long long)r;
            }
            run_add<unsigned long long, unsigned long long>(b, G, hg);
        }
    }
    flush_bins(hg, sumG, nb);
    if (bad) atomicAdd(inexact, bad);
}

// Vectors per bin (independent of the state; once per context).
__global__ void __launch_bounds__(RAD_THREADS) k_radial_count(int L, int nb, unsigned long long *count)
{
    extern __shared__ unsigned long long hc[];
    zero_bins(hc, nb);
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x; row < L * L; row += gridDim.x) {
        const int dy = min_image(row % L, L), dz = min_image(row / L, L);
        const int dyz = dy * dy + dz * dz;
        for (int x0 = threadIdx.x & ~31; x0 < L; x0 += blockDim.x) {
            const int x = x0 + lane;
            int b = -1;
            if (x < L) {
                const int dx = min_image(x, L);
                b = bin_of(dx * dx + dyz);
            }
            run_add<unsigned long long, unsigned long long>(b, b >= 0 ? 1ull : 0ull, hc);
        }
    }
    flush_bins(hc, count, nb);
}

// 6. out = [C(0..nb-1), S(0..nb-1), l]; cnt = [n_b (nb), inexact lags].
__global__ void k_radial_finish(int L, int nb, double c, const unsigned long long *sumG, const double *sumS,
                                const unsigned long long *count, const unsigned long long *inexact, double *out,
                                int64_t *cnt)
{
    const double N = (double)L * (double)L * (double)L;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double denom = __dmul_rn(N, (double)count[b]);
        out[b] = count[b] ? __ddiv_rn((double)(long long)sumG[b], denom) : 0.0;
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
        cnt[nb] = (int64_t)*inexact;
    }
}

// ---------------------------------------------------------------------------------
struct RadialPlans {
    int L = 0;
    bool made[2] = {false, false};
    cufftHandle fwd[2] = {0, 0}, inv[2] = {0, 0};
    size_t work[2] = {0, 0};
    char *buf = nullptr;  // transform buffer (grown to the largest precision used)
    size_t buf_bytes = 0;
    char *wk = nullptr;   // cuFFT work area
    size_t wk_bytes = 0;
    unsigned long long *count = nullptr;  // vectors per bin (counted at the first call)
    char *acc = nullptr;                  // per-call sums: sumG, sumS, inexact
};

RadialPlans *radial_plans_create() { return new (std::nothrow) RadialPlans(); }

void radial_release(RadialPlans *p, cudaStream_t s)
{
    if (!p) return;
    if (p->buf) cudaFreeAsync(p->buf, s);
    if (p->wk) cudaFreeAsync(p->wk, s);
    p->buf = p->wk = nullptr;
    p->buf_bytes = p->wk_bytes = 0;
}

void radial_plans_destroy(RadialPlans *p, cudaStream_t s)
{
    if (!p) return;
    radial_release(p, s);
    if (p->count) cudaFreeAsync(p->count, s);
    if (p->acc) cudaFreeAsync(p->acc, s);
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

// Grow a cached device allocation to at least `bytes` (stream-ordered).
static cudaError_t ensure(char **ptr, size_t *have, size_t bytes, cudaStream_t s)
{
    if (*have >= bytes && (*ptr || bytes == 0)) return cudaSuccess;
    if (*ptr) cudaFreeAsync(*ptr, s);
    *ptr = nullptr;
    *have = 0;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMallocAsync((void **)ptr, bytes, s);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return e;
    }
    *have = bytes;
    return cudaSuccess;
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
    cudaError_t e;
    if ((e = ensure(&p->buf, &p->buf_bytes, radial_scratch_bytes(L, prec), s)) != cudaSuccess) return e;
    if ((e = ensure(&p->wk, &p->wk_bytes, p->work[prec], s)) != cudaSuccess) return e;
    const size_t acc_bytes = (size_t)nb * 2 * sizeof(double) + 64;
    if (!p->acc && (e = cudaMallocAsync((void **)&p->acc, acc_bytes, s)) != cudaSuccess) {
        p->acc = nullptr;
        return e;
    }
    unsigned long long *sumG = reinterpret_cast<unsigned long long *>(p->acc);
    double *sumS = reinterpret_cast<double *>(p->acc) + nb;
    unsigned long long *inexact = reinterpret_cast<unsigned long long *>(p->acc) + 2 * nb;
    if ((e = cudaMemsetAsync(p->acc, 0, acc_bytes, s)) != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)(sms * 4);
    const size_t smem = (size_t)nb * sizeof(double);
    if (!p->count) {
        if ((e = cudaMallocAsync((void **)&p->count, sizeof(unsigned long long) * nb, s)) != cudaSuccess) {
            p->count = nullptr;
            return e;
        }
        if ((e = cudaMemsetAsync(p->count, 0, sizeof(unsigned long long) * nb, s)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_radial_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_radial_count<<<grid, RAD_THREADS, smem, s>>>(L, nb, p->count);
        if (launches) *launches += 1;
    }

    k_unpack_real<T><<<grid, RAD_THREADS, 0, s>>>(lat_r, reinterpret_cast<T *>(p->buf), g, P);
    cufftHandle f = p->fwd[prec], iv = p->inv[prec];
    if ((cs = cufftSetStream(f, s)) != CUFFT_SUCCESS || (cs = cufftSetStream(iv, s)) != CUFFT_SUCCESS ||
        (cs = cufftSetWorkArea(f, p->wk)) != CUFFT_SUCCESS || (cs = cufftSetWorkArea(iv, p->wk)) != CUFFT_SUCCESS) {
        *cufft_status = cs;
        return cudaErrorUnknown;
    }
    using C = typename Cx<T>::type;
    if (prec)
        cs = cufftExecD2Z(f, reinterpret_cast<cufftDoubleReal *>(p->buf), reinterpret_cast<cufftDoubleComplex *>(p->buf));
    else
        cs = cufftExecR2C(f, reinterpret_cast<cufftReal *>(p->buf), reinterpret_cast<cufftComplex *>(p->buf));
    if (cs != CUFFT_SUCCESS) {
        *cufft_status = cs;
        return cudaErrorUnknown;
    }
    if ((e = cudaFuncSetAttribute(k_power<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    k_power<T><<<grid, RAD_THREADS, smem, s>>>(reinterpret_cast<C *>(p->buf), L, nb, sumS);
    if (prec)
        cs = cufftExecZ2D(iv, reinterpret_cast<cufftDoubleComplex *>(p->buf), reinterpret_cast<cufftDoubleReal *>(p->buf));
    else
        cs = cufftExecC2R(iv, reinterpret_cast<cufftComplex *>(p->buf), reinterpret_cast<cufftReal *>(p->buf));
    if (cs != CUFFT_SUCCESS) {
        *cufft_status = cs;
        return cudaErrorUnknown;
    }
    const double invN = 1.0 / ((double)L * (double)L * (double)L);  // exact: N is a power of two
    if ((e = cudaFuncSetAttribute(k_radial_corr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    k_radial_corr<T><<<grid, RAD_THREADS, smem, s>>>(reinterpret_cast<const T *>(p->buf), L, P, nb, invN, sumG,
                                                       inexact);
    k_radial_finish<<<1, 256, 0, s>>>(L, nb, c, sumG, sumS, p->count, inexact, out, cnt);
    if (launches) *launches += 4;  // own kernels; the two cuFFT executions are library launches
    return cudaGetLastError();
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
