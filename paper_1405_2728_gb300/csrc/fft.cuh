// Shared-memory FFT building blocks for the zero-padded demagnetisation
// convolution (the "FFT accelerated convolution" of Section 3).
//
// A row of L = 2^l complex values lives in shared memory and is transformed
// in place by G = max(1, L/8) threads with self-sorting Stockham passes
// (Stockham; Cochran et al., Proc. IEEE 55 (1967) 1664): an optional first
// pass of radix 2 or 4 and then radix-8 passes.  Each thread keeps one radix-8
// butterfly (or two radix-4 / four radix-2 ones) in registers per pass; a
// barrier separates the loads of a pass from its stores, which makes the
// in-place update safe.  Twiddles come from a table tw[t] = exp(-2 pi i t/L')
// read with stride ts = L'/L.
//
// Zero padding is exploited where the convolution needs it:
//  HALF_IN : the upper half of the input is known to be zero, so the first
//            pass reads half of its inputs and skips the arithmetic on zeros;
//  HALF_OUT: only the lower half of the output is wanted, so the last pass
//            computes and stores only those values.
#pragma once

#include "common.cuh"

template <typename V> __device__ __forceinline__ V czero() { V r; r.x = 0; r.y = 0; return r; }

// Rows in shared memory are stored with one padding element after every 8:
// element i lives at pidx(i).  Stockham stores of radix 8 and strides 1 or 8
// then spread over all banks instead of hitting one bank group.
__host__ __device__ __forceinline__ int pidx(int i) { return i + (i >> 3); }
// shared-memory footprint (elements) of a padded row of length L, plus one
// element so that consecutive rows start in different banks
__host__ __device__ __forceinline__ int padded_row(int L) { return L + (L >> 3) + 1; }

// Row layout by element size.  16-byte elements (double2) use the padding
// above: each Stockham pass then takes the minimum number of shared-memory
// wavefronts.  8-byte elements (float2) are served 16 per wavefront; with
// the padding a warp's 32 consecutive elements span 36 slots, which costs 3
// to 4 wavefronts instead of 2.  They use an XOR swizzle instead, within
// aligned groups of 16 elements: bits 4-6 of the index are XORed into
// bits 0-3 (bit 6 into bit 3).  In a bank simulation of the radix-8
// Stockham passes this keeps unit-stride loads, the stride-8 stores of the
// first pass and the grouped stores of the later passes at 2 wavefronts
// (L = 512, 4096).  It is a permutation of every aligned group of 16, so a
// row of L elements needs only L slots, plus one between rows.
template <typename V> __host__ __device__ __forceinline__ int spos(int i)
{
    if constexpr (sizeof(V) == 8) return i ^ (((i >> 4) & 7) | (((i >> 6) & 1) << 3));
    else return i + (i >> 3);
}
__host__ __device__ __forceinline__ int row_stride(int L, int esz)
{
    return esz == 8 ? L + 1 : padded_row(L);
}

// copy a twiddle table of n complex values into shared memory (all threads)
template <typename V> __device__ __forceinline__ void load_twiddles(V *dst, const V *src, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// the same, issued as asynchronous copies (8 or 16 bytes per element);
// complete at cp_async_wait_all() of each thread, then a barrier
template <typename V> __device__ __forceinline__ void load_twiddles_async(V *dst, const V *src, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if constexpr (sizeof(V) == 16) cp_async16(dst + i, src + i);
        else cp_async8(dst + i, src + i);
    }
}

// 2-point DFT
template <bool HIN, typename V> __device__ __forceinline__ void dft2(V &a0, V &a1)
{
    if (HIN) { a1 = a0; return; }
    V t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

// 4-point DFT, forward uses -i, inverse +i; outputs in natural order
template <bool INV, bool HIN, typename V> __device__ __forceinline__ void dft4(V &x0, V &x1, V &x2, V &x3)
{
    V t0, t1, t2, t3;
    if (HIN) {           // x2 = x3 = 0
        t0 = x0; t1 = x0; t2 = x1; t3 = cmul_mi<INV>(x1);
    } else {
        t0 = cadd(x0, x2); t1 = csub(x0, x2);
        t2 = cadd(x1, x3); t3 = cmul_mi<INV>(csub(x1, x3));
    }
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

// 8-point DFT by one radix-2 decimation-in-frequency split into two 4-point
// DFTs: u_n = a_n + a_{n+4}, v_n = (a_n - a_{n+4}) W^n, X_{2k} = DFT4(u)_k,
// X_{2k+1} = DFT4(v)_k, W = exp(-+ i pi/4).
template <bool INV, bool HIN, typename V> __device__ __forceinline__ void dft8(V *a)
{
    typedef decltype(a[0].x) T;
    const T r = (T)0.70710678118654752440084436210484903928;
    V u0, u1, u2, u3, d0, d1, d2, d3;
    if (HIN) {
        u0 = a[0]; u1 = a[1]; u2 = a[2]; u3 = a[3];
        d0 = a[0]; d1 = a[1]; d2 = a[2]; d3 = a[3];
    } else {
        u0 = cadd(a[0], a[4]); d0 = csub(a[0], a[4]);
        u1 = cadd(a[1], a[5]); d1 = csub(a[1], a[5]);
        u2 = cadd(a[2], a[6]); d2 = csub(a[2], a[6]);
        u3 = cadd(a[3], a[7]); d3 = csub(a[3], a[7]);
    }
    V v1, v2, v3;
    if (INV) {
        v1.x = r * (d1.x - d1.y); v1.y = r * (d1.x + d1.y);
        v2.x = -d2.y;             v2.y = d2.x;
        v3.x = -r * (d3.x + d3.y); v3.y = r * (d3.x - d3.y);
    } else {
        v1.x = r * (d1.x + d1.y); v1.y = r * (d1.y - d1.x);
        v2.x = d2.y;              v2.y = -d2.x;
        v3.x = r * (d3.y - d3.x); v3.y = -r * (d3.x + d3.y);
    }
    dft4<INV, false>(u0, u1, u2, u3);
    dft4<INV, false>(d0, v1, v2, v3);
    a[0] = u0; a[1] = d0; a[2] = u1; a[3] = v1;
    a[4] = u2; a[5] = v2; a[6] = u3; a[7] = v3;
}

template <int R, bool INV, bool HIN, typename V> __device__ __forceinline__ void dftR(V *a)
{
    if (R == 2) dft2<HIN>(a[0], a[1]);
    else if (R == 4) dft4<INV, HIN>(a[0], a[1], a[2], a[3]);
    else dft8<INV, HIN>(a);
}

// One Stockham pass of radix R over a row of length L (Ns = product of the
// radices of the previous passes).  Thread j handles butterflies j + q G,
// q < 8/R.  Caller guarantees visibility of the row before the call; the
// pass ends with a barrier.
//
// Padded offsets in closed form (Ns, R, LR = L/R powers of two): butterfly b
// reads elements b + r LR, whose padded offsets are pidx(b) + r (LR + LR/8)
// when 8 divides LR; it writes elements (b - k) R + k + r Ns, k = b mod Ns,
// whose padded offsets are 9 (b - k) + k + k/8 + r Ns + (r Ns)/8 for R = 8
// (and likewise with (b - k) R for R < 8), since k < Ns and Ns divides or is
// a multiple of 8.
template <int R, bool INV, bool HIN, bool HOUT, typename V>
__device__ __forceinline__ void stockham_pass(V *row, int L, int Ns, int j, int G,
                                              const V *__restrict__ tw, int ts, bool active)
{
    constexpr int NB = 8 / R;
    V v[8];
    const int LR = L / R;
    const int ld9 = LR + (LR >> 3);       // padded stride between the inputs of a butterfly (8 | LR)
    const int tstep0 = (L / (Ns * R)) * ts;
    if (active) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int b = j + q * G;
            const int p0 = pidx(b);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (HIN && r >= R / 2) { v[q * R + r] = czero<V>(); continue; }
                if constexpr (sizeof(V) == 8) v[q * R + r] = row[spos<V>(b + r * LR)];
                else v[q * R + r] = row[(LR & 7) ? pidx(b + r * LR) : p0 + r * ld9];
            }
            if (Ns > 1) {
                const int step = tstep0 * (b & (Ns - 1));
                int t = step;
#pragma unroll
                for (int r = 1; r < R; ++r, t += step) {
                    const V w = tw[t];
                    v[q * R + r] = INV ? cmulc(v[q * R + r], w) : cmul(v[q * R + r], w);
                }
            }
            dftR<R, INV, HIN>(&v[q * R]);
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int b = j + q * G;
            const int k = b & (Ns - 1);
            const int hi = (b - k) * R;                  // multiple of 8 when R == 8
            const int s0 = (R == 8) ? hi + (hi >> 3) + k + (k >> 3) : 0;
#pragma unroll
            for (int r = 0; r < (HOUT ? R / 2 : R); ++r) {
                const int rn = r * Ns;
                if constexpr (sizeof(V) == 8) row[spos<V>(hi + k + rn)] = v[q * R + r];
                else row[(R == 8) ? s0 + rn + (rn >> 3) : pidx(hi + k + rn)] = v[q * R + r];
            }
        }
    }
    __syncthreads();
}

// In-place FFT of one shared-memory row of length L = 2^logL (forward:
// exp(-i...), inverse: exp(+i...), unnormalised).  Every thread of the CTA
// must call this with the same L (it contains barriers); thread j in [0, G)
// of the row's group works on it.  Threads with active == false (padding
// threads of the CTA) only take part in the barriers.  The caller
// synchronises before the call so that the row's contents are visible; the
// row is final after return.  Twiddles: tw[t * TS] = exp(-2 pi i t / L).
//
// fft_row_n takes L at run time; fft_row_c<LOGL> is the same sequence of
// passes with L a compile-time constant, so that every offset, stride and
// pass count folds into the instructions.  Kernels are instantiated for the
// common lengths (template parameter LC of fft_row) and the host launches
// the matching instance.
template <bool INV, bool HIN, bool HOUT, int TS, typename V>
__device__ __forceinline__ void fft_row_n(V *row, int L, int logL, int j, const V *__restrict__ tw, bool active)
{
    if (L == 1) return;
    if (L < 8) {
        // G == 1: the single thread of the row does the whole transform.  The
        // barriers stay outside the branches so that every thread of a warp
        // executes the same barrier instruction.
        V a[4];
        if (active) {
            a[0] = row[0];
            a[1] = (HIN && L == 2) ? czero<V>() : row[1];
            if (L == 2) {
                dft2<HIN>(a[0], a[1]);
            } else {
                a[2] = HIN ? czero<V>() : row[2];
                a[3] = HIN ? czero<V>() : row[3];
                dft4<INV, HIN>(a[0], a[1], a[2], a[3]);
            }
        }
        __syncthreads();
        if (active) {
            row[0] = a[0];
            if (L == 2) {
                if (!HOUT) row[1] = a[1];
            } else {
                row[1] = a[1];
                if (!HOUT) { row[2] = a[2]; row[3] = a[3]; }
            }
        }
        __syncthreads();
        return;
    }
    const int G = L >> 3;
    const int rem = logL % 3;
    const int n8 = logL / 3;
    int Ns = 1;
    bool first = true;
    if (rem == 1) {
        stockham_pass<2, INV, HIN, false>(row, L, Ns, j, G, tw, TS, active);
        Ns = 2; first = false;
    } else if (rem == 2) {
        stockham_pass<4, INV, HIN, false>(row, L, Ns, j, G, tw, TS, active);
        Ns = 4; first = false;
    }
    for (int p = 0; p < n8; ++p) {
        const bool last = (p == n8 - 1);
        if (first && HIN) {
            if (last && HOUT) stockham_pass<8, INV, true, true>(row, L, Ns, j, G, tw, TS, active);
            else stockham_pass<8, INV, true, false>(row, L, Ns, j, G, tw, TS, active);
        } else {
            if (last && HOUT) stockham_pass<8, INV, false, true>(row, L, Ns, j, G, tw, TS, active);
            else stockham_pass<8, INV, false, false>(row, L, Ns, j, G, tw, TS, active);
        }
        Ns <<= 3;
        first = false;
    }
}

template <int LOGL, bool INV, bool HIN, bool HOUT, int TS, typename V>
__device__ __forceinline__ void fft_row_c(V *row, int j, const V *__restrict__ tw, bool active)
{
    static_assert(LOGL >= 3, "compile-time rows have at least 8 elements");
    constexpr int L = 1 << LOGL, G = L >> 3, rem = LOGL % 3, n8 = LOGL / 3;
    constexpr int NS0 = rem == 1 ? 2 : (rem == 2 ? 4 : 1);
    if constexpr (rem == 1) stockham_pass<2, INV, HIN, false>(row, L, 1, j, G, tw, TS, active);
    if constexpr (rem == 2) stockham_pass<4, INV, HIN, false>(row, L, 1, j, G, tw, TS, active);
#pragma unroll
    for (int p = 0; p < n8; ++p) {
        const int Ns = NS0 << (3 * p);
        const bool last = (p == n8 - 1), first = (p == 0 && rem == 0);
        if (first && HIN) {
            if (last && HOUT) stockham_pass<8, INV, true, true>(row, L, Ns, j, G, tw, TS, active);
            else stockham_pass<8, INV, true, false>(row, L, Ns, j, G, tw, TS, active);
        } else {
            if (last && HOUT) stockham_pass<8, INV, false, true>(row, L, Ns, j, G, tw, TS, active);
            else stockham_pass<8, INV, false, false>(row, L, Ns, j, G, tw, TS, active);
        }
    }
}

// LC > 0: the kernel was compiled for rows of length 2^LC (L, logL unused);
// LC == 0: any length
template <bool INV, bool HIN, bool HOUT, int TS, int LC, typename V>
__device__ __forceinline__ void fft_row(V *row, int L, int logL, int j, const V *__restrict__ tw, bool active)
{
    if constexpr (LC > 0) fft_row_c<LC, INV, HIN, HOUT, TS>(row, j, tw, active);
    else fft_row_n<INV, HIN, HOUT, TS>(row, L, logL, j, tw, active);
}

// Row lengths with compiled specialisations in the field kernels (log2 of
// 64 .. 1024); other lengths take the generic code.
#define MM_FFT_SPECIALISED(logL) ((logL) >= 6 && (logL) <= 10)
