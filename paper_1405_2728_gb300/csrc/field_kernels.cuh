// Field kernels of one H_eff evaluation (and of the minimiser iteration),
// written as device bodies parameterised by the CTA's coordinates and its
// number of working threads, plus the single-problem kernels that call them.
// Included by heff.cu (single problems) and batch.cu (grouped launches over
// many problems), so both run the same arithmetic.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fft.cuh"

namespace {

template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ dfloat ldg(const dfloat *p)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return dfloat(v.x, v.y);
}
// complex loads through the read-only path (ld_nc) or cached in L2 only (ld_cg)
template <typename V> __device__ __forceinline__ V ld_nc(const V *p) { return __ldg(p); }
template <> __device__ __forceinline__ dcomplex ld_nc(const dcomplex *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return dcomplex{dfloat(v.x, v.y), dfloat(v.z, v.w)};
}
template <typename V> __device__ __forceinline__ V ld_cg(const V *p) { return __ldcg(p); }
template <> __device__ __forceinline__ dcomplex ld_cg(const dcomplex *p)
{
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    return dcomplex{dfloat(v.x, v.y), dfloat(v.z, v.w)};
}
// a value of the FFT arithmetic F read back in the field type T
template <typename T, typename F> __device__ __forceinline__ T to_field(F v) { return (T)v; }
template <> __device__ __forceinline__ double to_field<double, dfloat>(dfloat v) { return df_to_double(v); }
// a caller's value (double for double-word fields) in the field type T, and back
template <typename T> __device__ __forceinline__ T from_io(typename io_of<T>::type v) { return (T)v; }
template <typename T> __device__ __forceinline__ typename io_of<T>::type to_io(T v) { return v; }
template <> __device__ __forceinline__ double to_io<dfloat>(dfloat v) { return df_to_double(v); }
// 1/sqrt(x) in the field type (the double and float steps divide by sqrt)
template <typename T> __device__ __forceinline__ T inv_sqrt(T x) { return (T)1 / sqrt(x); }
template <> __device__ __forceinline__ dfloat inv_sqrt<dfloat>(dfloat x) { return df_rsqrt(x); }
// 1/|m| of the renormalisation after a midpoint step (float: the fast
// reciprocal square root, ~2 ulp; double-word: one Newton step, ~2^-47)
__device__ __forceinline__ float renorm_scale(float s) { return rsqrtf(s); }
__device__ __forceinline__ dfloat renorm_scale(dfloat s) { return df_rsqrt(s); }

// real element x of a padded complex row holding Px reals
template <typename T, typename V> __device__ __forceinline__ T &rel(V *row, int x)
{
    return reinterpret_cast<T *>(row + spos<V>(x >> 1))[x & 1];
}

// Rows of a field [3][nz][ny][nx] copied asynchronously into shared memory:
// dst [3][nrows][nx] receives rows y = ylo .. ylo + nrows - 1 of plane z
// (rows outside 0..ny-1 are skipped) in 16-byte chunks (the planner checked
// that rows start on 16-byte boundaries).
template <typename T>
__device__ __forceinline__ void stage_rows(T *dst, const T *__restrict__ src, const Geom &g, int z, int ylo,
                                           int nrows, int tid, int nth)
{
    constexpr int CH = 16 / sizeof(T);
    const int nx = g.nx, nc = g.fd_nc.d;
    const int tot = 3 * nrows * nc;
    const long plane = (long)z * g.ny * nx;
    if (tid >= nth) return;
    for (int q = tid; q < tot; q += nth) {
        const int rr = g.fd_nc.div(q), ch = q - rr * nc;  // rr = c * nrows + r
        const int c = (rr >= nrows) + (rr >= 2 * nrows), r = rr - c * nrows, y = ylo + r;
        if (y < 0 || y >= g.ny) continue;
        cp_async16(dst + (long)rr * nx + ch * CH, src + c * g.N + plane + (long)y * nx + ch * CH);
    }
}

// byte offset of the staging area of k_xinv (after the FFT rows and the
// twiddles, 16-byte aligned); it holds (15 TY + 6) rows of nx values
template <typename T> __host__ __device__ __forceinline__ size_t stage_offset(const Geom &g)
{
    return ((size_t)(3 * g.TY * g.rsx + g.Px) * 2 * sizeof(T) + 15) & ~(size_t)15;
}

// ---------------------------------------------------------------------------
// k_xfwd
// ---------------------------------------------------------------------------
// The kernel bodies take the CTA's coordinates and its number of working
// threads nth as arguments: a single problem launches them with its own
// grid (nth = blockDim.x); a batch launches one grid over the work items of
// many problems with blockDim.x the largest nth, and the threads at or above
// a problem's nth only take part in the barriers.  Loops start at tt, the
// thread index, or past every bound for those idle threads.
#define MM_IDLE_START (1 << 30)
template <typename T, typename F, bool MIN, int LX>
__device__ __forceinline__ void xfwd_body(const Geom &g, const FieldPtrs<T, F> &P, const int tid, const int nth,
                                          const int bx, const int by)
{
    typedef typename cvec<F>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tt = tid < nth ? tid : MM_IDLE_START;
    const int TY = g.TYF, y0 = bx * TY, z = by;
    const int nx = g.nx, ny = g.ny, Px = g.Px;
    const long N = g.N;
    V *tw = S + 3 * TY * g.rsx;  // Px twiddles exp(-2 pi i t / Px)
    for (int i = tt; i < Px; i += nth) tw[i] = P.tw_px[i];

    typedef typename io_of<T>::type IO;
    const T *src = nullptr;        // minimiser mode: the iterate buffers
    const IO *src_io = nullptr;    // otherwise the caller's m
    T *dst = nullptr;
    const T *gp = nullptr;
    T tau = 0;
    int step_kind = 0;
    if (MIN) {
        const MinState *st = P.st;
        const long k = st->k;
        const int cur = st->base ^ (int)(k & 1);
        if (k > 0) {
            src = cur ? P.mbuf[0] : P.mbuf[1];
            dst = cur ? P.mbuf[1] : P.mbuf[0];
            gp = ((k - 1) & 1) ? P.gbuf[1] : P.gbuf[0];
            tau = pick<T>(st->tau, st->tauf, st->tauw);
            step_kind = st->step_kind;
        } else {
            src = cur ? P.mbuf[1] : P.mbuf[0];
        }
    } else {
        src_io = P.m_src;
    }
    // load (and step) the tile; row (c, yl) holds Px reals
#pragma unroll(sizeof(T) == 4 ? 2 : 1)
    for (int e = tt; e < TY * nx; e += nth) {
        const int yl = g.fd_nx.div(e), x = e - yl * nx, y = y0 + yl;
        T m0 = 0, m1 = 0, m2 = 0;
        if (y < ny) {
            const long n = ((long)z * ny + y) * nx + x;
            if constexpr (MIN) {
                m0 = ldg(src + n); m1 = ldg(src + N + n); m2 = ldg(src + 2 * N + n);
            } else {
                m0 = from_io<T>(ldg(src_io + n)); m1 = from_io<T>(ldg(src_io + N + n));
                m2 = from_io<T>(ldg(src_io + 2 * N + n));
            }
            if (MIN && dst) {
                const T g0 = ldg(gp + n), g1 = ldg(gp + N + n), g2 = ldg(gp + 2 * N + n);
                if (step_kind == MM_STEP_CAYLEY) {
                    const T q = (T)0.25 * tau * tau * (g0 * g0 + g1 * g1 + g2 * g2);
                    const T a = (T)1 - q, inv = (T)1 / ((T)1 + q);
                    m0 = (a * m0 - tau * g0) * inv;
                    m1 = (a * m1 - tau * g1) * inv;
                    m2 = (a * m2 - tau * g2) * inv;
                    if constexpr (!std::is_same<T, double>::value) {
                        // the closed form keeps |m| = 1 exactly in exact arithmetic;
                        // its rounding drifts ~1e-7 per step in float and ~1e-14 in
                        // double-word arithmetic, so those paths renormalise (the
                        // double path keeps the pure midpoint form, ~1e-16 per step)
                        const T r = renorm_scale(m0 * m0 + m1 * m1 + m2 * m2);
                        m0 *= r; m1 *= r; m2 *= r;
                    }
                } else {
                    m0 -= tau * g0; m1 -= tau * g1; m2 -= tau * g2;
                    const T inv = inv_sqrt(m0 * m0 + m1 * m1 + m2 * m2);
                    m0 *= inv; m1 *= inv; m2 *= inv;
                }
                dst[n] = m0; dst[N + n] = m1; dst[2 * N + n] = m2;
            }
        }
        rel<F>(S + (0 * TY + yl) * g.rsx, x) = F(m0);
        rel<F>(S + (1 * TY + yl) * g.rsx, x) = F(m1);
        rel<F>(S + (2 * TY + yl) * g.rsx, x) = F(m2);
    }
    const int npad = Px - nx;
    for (int e = tt; e < 3 * TY * npad; e += nth) {
        const int row = g.fd_padx.div(e), x = nx + (e - row * npad);
        rel<F>(S + row * g.rsx, x) = F(0);
    }
    __syncthreads();

    // complex FFT of length Hx of the packed rows (upper half zero)
    {
        const int row = tid / g.Gx, j = tid - row * g.Gx;
        const bool act = row < 3 * TY;
        fft_row<false, true, false, 2, LX>(S + (act ? row : 0) * g.rsx, g.Hx, g.lhx, j, tw, act);
    }

    // unpack to the real-input spectrum X[k], k = 0..Hx, and store transposed.
    // With sum = Z[k] + Z*[Hx-k], dif = Z[k] - Z*[Hx-k] and w = exp(-2 pi i k / Px):
    // X[k] = (sum - i w dif) / 2 and, from the same two values (w^Hx = -1),
    // X[Hx-k] = (sum* - i (w dif)*) / 2; one item per pair k = 0..Hx/2.
    const int Hx = g.Hx, hh = Hx >> 1;
    for (int e = tt; e < TY * 3 * (hh + 1); e += nth) {
        const int c = e % 3, rest = e / 3, yl = rest & (TY - 1), k = rest >> g.ltyf;
        const int y = y0 + yl;
        const V *row = S + (c * TY + yl) * g.rsx;
        const V Zk = row[spos<V>(k)];
        const V Zm = cconj(row[spos<V>(k == 0 ? 0 : Hx - k)]);
        const V sum = cadd(Zk, Zm), dif = csub(Zk, Zm);
        const V wd = cmul(tw[k], dif);
        if (y < ny) {
            V X;
            X.x = F(0.5) * (sum.x + wd.y);
            X.y = F(0.5) * (sum.y - wd.x);
            P.W[(((long)k * g.nz + z) * ny + y) * 3 + c] = X;
            if (Hx - k != k) {
                X.x = F(0.5) * (sum.x - wd.y);
                X.y = F(0.5) * (-sum.y - wd.x);
                P.W[(((long)(Hx - k) * g.nz + z) * ny + y) * 3 + c] = X;
            }
        }
    }
}

template <typename T, typename F, bool MIN, int LX>
__global__ void __launch_bounds__(768) k_xfwd(Geom g, FieldPtrs<T, F> P)
{
    xfwd_body<T, F, MIN, LX>(g, P, threadIdx.x, blockDim.x, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// k_yz
// ---------------------------------------------------------------------------
// the double kernel runs fewer, fatter threads (its z-phase keeps ~100
// doubles live); the y rows are then transformed in batches of RB rows
template <typename T> struct YZBound { static constexpr int v = sizeof(T) == 8 ? 512 : 768; };

template <typename T, typename F, int PZ, int LY>
__device__ __forceinline__ void yz_body(const Geom &g, const FieldPtrs<T, F> &P, const int tid, const int nth,
                                        const int kx)
{
    typedef typename cvec<F>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tt = tid < nth ? tid : MM_IDLE_START;
    const int ny = g.ny, nz = g.nz, Py = g.Py;
    const int nrow = 3 * nz;
    V *Wk = P.W + (long)kx * nrow * ny;
    // Py twiddles: a shared copy in float; the double kernel reads them from
    // global memory (L1), which keeps its shared memory within two CTAs per SM
    const V *tw;
    if constexpr (sizeof(V) == 8) {
        V *tws = S + nrow * g.rsy;
        for (int i = tt; i < Py; i += nth) cp_async8(tws + i, P.tw_py + i);
        tw = tws;
    } else {
        tw = P.tw_py;
    }

    // Wk[z][y][c] -> row (c, z); PF loads per thread in flight before use
    constexpr int PF = sizeof(V) == 8 ? 8 : 4;
    const int tot = nrow * ny;
    for (int e0 = tt; e0 < tot; e0 += PF * nth) {
        V v[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e < tot) v[i] = ld_cg(Wk + e);
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e >= tot) break;
            const int c = e % 3, rest = e / 3, zz = g.fd_ny.div(rest), y = rest - zz * ny;
            S[(c * nz + zz) * g.rsy + spos<V>(y)] = v[i];
        }
    }
    const int npad = Py - ny;
    for (int e = tt; e < nrow * npad; e += nth) {
        const int row = g.fd_pady.div(e), y = ny + (e - row * npad);
        S[row * g.rsy + spos<V>(y)] = czero<V>();
    }
    cp_async_wait_all();
    __syncthreads();
    const int rb = tid / g.Gy, j = tid - rb * g.Gy;  // row within a batch of g.RB rows
    const bool act = rb < g.RB;
    for (int r0 = 0; r0 < nrow; r0 += g.RB)
        fft_row<false, true, false, 1, LY>(S + (act ? r0 + rb : 0) * g.rsy, Py, g.lpy, j, tw, act);

    // per ky: the z direction as a direct convolution (films have nz <= 4).
    // With the tensor transformed along x and y only, K(kx, ky, dz), the
    // field is H^_a(z) = sum_b sum_z' K_ab(z - z') m^_b(z') -- the same sums
    // the zero-padded z-FFT, product and inverse z-FFT would form, in fewer
    // operations and with no twiddles.  K_xx, K_yy, K_zz, K_xy are real and
    // even in dz, K_xz and K_yz imaginary and odd in dz (and zero at dz = 0);
    // K_xy, K_yz are odd in ky.  Stored for dz = 0 .. NZM-1 (zero beyond
    // nz - 1, so that every load is unconditional) as
    // [kx][dz][component][ky <= Py/2], scaled by -Ms/(Px Py).
    constexpr int NZM = PZ > 1 ? PZ / 2 : 1;  // nz <= NZM
    const int hy = Py / 2, kst = hy + 1;
    const F *Kk = P.Nhat + (long)kx * NZM * 6 * kst;
    for (int ky = tt; ky < Py; ky += nth) {
        const int pky = spos<V>(ky);
        const int kyr = ky <= hy ? ky : Py - ky;
        const bool flip = ky > hy;
        V mz[3][NZM], hz[3][NZM];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int n = 0; n < NZM; ++n) {
                mz[c][n] = (n < nz) ? S[(c * nz + n) * g.rsy + pky] : czero<V>();
                hz[c][n] = czero<V>();
            }
#pragma unroll
        for (int dz = 0; dz < NZM; ++dz) {
            const F *kd = Kk + (long)dz * 6 * kst + kyr;
            const F kxx = ldg(kd), kyy = ldg(kd + kst), kzz = ldg(kd + 2 * kst);
            const F kxy0 = ldg(kd + 3 * kst), kxz = ldg(kd + 4 * kst), kyz0 = ldg(kd + 5 * kst);
            const F kxy = flip ? -kxy0 : kxy0, kyz = flip ? -kyz0 : kyz0;
#pragma unroll
            for (int z = 0; z < NZM; ++z)
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    // source z' = z - dz (side 0) or z + dz (side 1); K(z - z') of the
                    // odd components is +K(dz) for z' < z and -K(dz) for z' > z
                    if (side == 1 && dz == 0) continue;
                    const int zp = side ? z + dz : z - dz;
                    if (zp < 0 || zp >= NZM) continue;
                    const V a = mz[0][zp], b = mz[1][zp], c = mz[2][zp];
                    hz[0][z].x += kxx * a.x + kxy * b.x; hz[0][z].y += kxx * a.y + kxy * b.y;
                    hz[1][z].x += kxy * a.x + kyy * b.x; hz[1][z].y += kxy * a.y + kyy * b.y;
                    hz[2][z].x += kzz * c.x;             hz[2][z].y += kzz * c.y;
                    if (dz > 0) {  // i * (+-k) * m = (-+k m.y, +-k m.x)
                        const F sxz = side ? -kxz : kxz, syz = side ? -kyz : kyz;
                        hz[0][z].x -= sxz * c.y;             hz[0][z].y += sxz * c.x;
                        hz[1][z].x -= syz * c.y;             hz[1][z].y += syz * c.x;
                        hz[2][z].x -= sxz * a.y + syz * b.y; hz[2][z].y += sxz * a.x + syz * b.x;
                    }
                }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int zz = 0; zz < NZM; ++zz)
                if (zz < nz) S[(c * nz + zz) * g.rsy + pky] = hz[c][zz];
    }
    __syncthreads();
    for (int r0 = 0; r0 < nrow; r0 += g.RB)
        fft_row<true, false, true, 1, LY>(S + (act ? r0 + rb : 0) * g.rsy, Py, g.lpy, j, tw, act);

    for (int e = tt; e < nrow * ny; e += nth) {
        const int c = e % 3, rest = e / 3, zz = g.fd_ny.div(rest), y = rest - zz * ny;
        Wk[e] = S[(c * nz + zz) * g.rsy + spos<V>(y)];
    }
}

template <typename T, typename F, int PZ, int LY>
__global__ void __launch_bounds__(YZBound<T>::v) k_yz(Geom g, FieldPtrs<T, F> P)
{
    yz_body<T, F, PZ, LY>(g, P, threadIdx.x, blockDim.x, blockIdx.x);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// Slots of the per-CTA partial sums.  In MODE_MIN: s.s, s.y, y.y,
// max |m x H|^2, energy density sum, sum m.  In MODE_ENERGY: m.H_demag,
// m.H_exchange, K(1 - (m.u)^2), m.H_ext, -, sum m.
enum { SL_SS = 0, SL_SY = 1, SL_YY = 2, SL_T2 = 3, SL_ET = 4, SL_MX = 5, SL_MY = 6, SL_MZ = 7, NSL = 8 };
enum { SL_ED = 0, SL_EEX = 1, SL_EAN = 2, SL_EZ = 3 };
static_assert(NSL <= RED_NSLOT, "partials buffer holds RED_NSLOT doubles per CTA");
static_assert(NSL % 2 == 0 && RED_NSLOT % 2 == 0, "the last CTA reads the partials in 16-byte pairs");

// accumulator: double on the double path, a compensated float pair on the float path
template <typename T> struct Acc;
template <> struct Acc<double> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void add_prod(double a, double b) { v += a * b; }
    __device__ __forceinline__ void add(const Acc &o) { v += o.v; }
    __device__ __forceinline__ void maxv(double x) { v = fmax(v, x); }
    __device__ __forceinline__ void maxv(const Acc &o) { v = fmax(v, o.v); }
    __device__ __forceinline__ Acc shfl_down(int o) const { Acc r; r.v = __shfl_down_sync(0xffffffffu, v, o); return r; }
    __device__ __forceinline__ double value() const { return v; }
};
template <> struct Acc<float> {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
    __device__ __forceinline__ void add(float x)
    {
        const float s = hi + x, bb = s - hi;
        lo += (hi - (s - bb)) + (x - bb);
        hi = s;
    }
    // a * b added exactly: the product is split into its rounded value and
    // the rounding error (exact with one FMA: Dekker's TwoProduct in the form
    // of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005) 1955)
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        add(p);
        lo += e;
    }
    __device__ __forceinline__ void add(const Acc &o) { add(o.hi); lo += o.lo; }
    __device__ __forceinline__ void maxv(float x) { hi = fmaxf(hi, x); }
    __device__ __forceinline__ void maxv(const Acc &o) { hi = fmaxf(hi, o.hi); }
    __device__ __forceinline__ Acc shfl_down(int o) const
    {
        Acc r;
        r.hi = __shfl_down_sync(0xffffffffu, hi, o);
        r.lo = __shfl_down_sync(0xffffffffu, lo, o);
        return r;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// double-word accumulator of the MM_F32X2 fields: per-cell products and sums
// in double-word arithmetic (relative rounding a few units of 2^-48 per
// operation), converted to double for the sums across CTAs
template <> struct Acc<dfloat> {
    dfloat v;
    __device__ __forceinline__ void zero() { v = dfloat(0.0f, 0.0f); }
    __device__ __forceinline__ void add(dfloat x) { v = v + x; }
    __device__ __forceinline__ void add_prod(dfloat a, dfloat b) { v = v + a * b; }
    __device__ __forceinline__ void add(const Acc &o) { v = v + o.v; }
    __device__ __forceinline__ void maxv(dfloat x)
    {
        if (x.hi > v.hi || (x.hi == v.hi && x.lo > v.lo)) v = x;
    }
    __device__ __forceinline__ void maxv(const Acc &o) { maxv(o.v); }
    __device__ __forceinline__ Acc shfl_down(int o) const
    {
        Acc r;
        r.v.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        r.v.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        return r;
    }
    __device__ __forceinline__ double value() const { return df_to_double(v); }
};

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Last CTA of the field evaluation: sum the per-CTA partials in block order
// (one warp; fixed order, so the result does not depend on which CTA came
// last), then finish the iteration on lane 0.
template <int MODE>
__device__ void finish_iteration(const Geom &g, double *partials, int nblk, MinState *st,
                                 cudaGraphConditionalHandle h, int use_cond, int body_kernels)
{
    const int lane = threadIdx.x & 31;
    // lane l sums blocks l, l + 32, l + 64, ... of every slot in that order;
    // the loads of FB blocks (all slots, 16-byte reads) are issued before any
    // is added, so the wait is one L2 round trip per FB blocks, not one per
    // block and slot
    constexpr int FB = 2;
    double v[NSL];
#pragma unroll
    for (int s = 0; s < NSL; ++s) v[s] = 0.0;
    auto fold = [&](const double2 *x) {
#pragma unroll
        for (int s = 0; s < NSL; ++s) {
            const double xs = (s & 1) ? x[s / 2].y : x[s / 2].x;
            v[s] = (MODE == MODE_MIN && s == SL_T2) ? fmax(v[s], xs) : v[s] + xs;
        }
    };
    int b = lane;
    for (; b + (FB - 1) * 32 < nblk; b += FB * 32) {
        double2 x[FB][NSL / 2];
#pragma unroll
        for (int i = 0; i < FB; ++i)
#pragma unroll
            for (int q = 0; q < NSL / 2; ++q)
                x[i][q] = __ldcg(reinterpret_cast<const double2 *>(partials + (long)(b + 32 * i) * RED_NSLOT) + q);
#pragma unroll
        for (int i = 0; i < FB; ++i) fold(x[i]);
    }
    for (; b < nblk; b += 32) {
        double2 x[NSL / 2];
#pragma unroll
        for (int q = 0; q < NSL / 2; ++q) x[q] = __ldcg(reinterpret_cast<const double2 *>(partials + (long)b * RED_NSLOT) + q);
        fold(x);
    }
    double tot[NSL];
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
        const bool isMax = (MODE == MODE_MIN && s == SL_T2);
        double w = v[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, w, o);
            w = isMax ? fmax(w, y) : w + y;
        }
        tot[s] = w;
    }
    if (lane != 0) return;
    const double V = g.dx * g.dy * g.dz, Ms = g.Ms, cE = MM_MU0 * Ms * V;
    st->mavg[0] = tot[SL_MX] / (double)g.N;
    st->mavg[1] = tot[SL_MY] / (double)g.N;
    st->mavg[2] = tot[SL_MZ] / (double)g.N;
    if (MODE == MODE_ENERGY) {
        const double Ed = -0.5 * cE * tot[SL_ED], Eex = -0.5 * cE * tot[SL_EEX];
        const double Ean = V * tot[SL_EAN], Ez = -cE * tot[SL_EZ];
        st->energy[0] = Ed; st->energy[1] = Eex; st->energy[2] = Ean; st->energy[3] = Ez;
        st->energy[4] = Ed + Eex + Ean + Ez;
        return;
    }
    const long k = st->k;
    const double tmax = sqrt(tot[SL_T2]);
    st->max_torque = tmax / Ms;
    st->bb[0] = k > 0 ? tot[SL_SS] : 0.0;
    st->bb[1] = k > 0 ? tot[SL_SY] : 0.0;
    st->bb[2] = k > 0 ? tot[SL_YY] : 0.0;
    st->energy[4] = cE * tot[SL_ET];
    st->evals = k + 1;
    st->launches += body_kernels;
    if (k == 0) st->t_start_ns = globaltimer_ns();
    int stop = 1;
    const bool finite = isfinite(tmax) && isfinite(st->energy[4]) &&
                        (k == 0 || (isfinite(tot[SL_SS]) && isfinite(tot[SL_SY]) && isfinite(tot[SL_YY])));
    if (!finite) {
        st->status = MMS_NONFINITE;
    } else if (tmax < st->tol_abs) {
        st->status = MMS_CONVERGED;
    } else if (k >= st->max_iter) {
        st->status = MMS_MAXITER;
    } else if (st->timeout_ns && globaltimer_ns() - st->t_start_ns > st->timeout_ns) {
        st->status = MMS_TIMEOUT;
    } else {
        double tau;
        if (k == 0) {
            tau = st->tau0;
        } else {
            const double ss = tot[SL_SS], sy = tot[SL_SY], yy = tot[SL_YY];
            if (st->tau_rule == MM_TAU_ADAPTIVE)   // tau^2 when cos^2(s, y) < kappa, else tau^1
                tau = (sy * sy < st->kappa * (ss * yy)) ? sy / yy : ss / sy;
            else                                   // alternation: tau^1 on odd k, tau^2 on even k
                tau = (k & 1) ? ss / sy : sy / yy;
            if (!(isfinite(tau) && tau > 0.0)) tau = sqrt(ss / yy);
            if (!(isfinite(tau) && tau > 0.0)) tau = st->tau0;
        }
        st->tau = tau;
        st->tauf = (float)tau;
        st->tauw = dfloat(tau);
        st->k = k + 1;
        stop = 0;
    }
    if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// k_xinv
// ---------------------------------------------------------------------------
// bid: this CTA's slot among the problem's nblk CTAs (partial sums, completion count)
template <typename T, typename F, int MODE, int LX>
__device__ __forceinline__ void xinv_body(const Geom &g, const FieldPtrs<T, F> &P, double hx0, double hx1, double hx2,
                                          cudaGraphConditionalHandle h, int use_cond, const int tid, const int nth,
                                          const int bx, const int by, const int bid, const int nblk)
{
    typedef typename cvec<F>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tt = tid < nth ? tid : MM_IDLE_START;
    const int TY = g.TY, y0 = bx * TY, z = by;
    const int nx = g.nx, ny = g.ny, nz = g.nz, Hx = g.Hx;
    const long N = g.N;
    V *tw = S + 3 * TY * g.rsx;

    MinState *st = P.st;
    long k = 0;
    int cur = 0;
    typedef typename io_of<T>::type IO;
    constexpr bool FROM_T = MODE == MODE_MIN || std::is_same<T, IO>::value;
    const T *m = nullptr;       // m in the field type (the iterate, or the caller's m of that type)
    const IO *mio = nullptr;    // the caller's m when it is of another type (converted per load)
    const T *mp = nullptr, *gq = nullptr;
    if (MODE == MODE_MIN) {
        k = st->k;
        cur = st->base ^ (int)(k & 1);
        m = cur ? P.mbuf[1] : P.mbuf[0];
        mp = cur ? P.mbuf[0] : P.mbuf[1];
        gq = (k & 1) ? P.gbuf[0] : P.gbuf[1];  // g_{k-1}
    } else if constexpr (std::is_same<T, IO>::value) {
        m = P.m_src;
    } else {
        mio = P.m_src;
    }
    auto mval = [&](long i) -> T {
        if constexpr (FROM_T) return m[i];
        else return from_io<T>(mio[i]);
    };
    // the float kernel stages the local terms' inputs -- m on planes z-1, z,
    // z+1 (rows y0-1 .. y0+TY on its own plane), m_{k-1} and g_{k-1} -- with
    // cp.async now; they arrive while the inverse x-FFT runs
    const bool stg = sizeof(T) == 4 && MODE == MODE_MIN && g.stage;
    T *SG = reinterpret_cast<T *>(smem_raw + stage_offset<T>(g));
    const int oZm = 3 * (TY + 2) * nx, oZp = oZm + 3 * TY * nx, oMP = oZp + 3 * TY * nx, oGQ = oMP + 3 * TY * nx;
    for (int i = tt; i < g.Px; i += nth) {
        if constexpr (sizeof(V) == 16) cp_async16(tw + i, P.tw_px + i);
        else cp_async8(tw + i, P.tw_px + i);
    }
    cp_async_commit();
    if (stg) {
        stage_rows(SG, m, g, z, y0 - 1, TY + 2, tid, nth);
        if (z > 0) stage_rows(SG + oZm, m, g, z - 1, y0, TY, tid, nth);
        if (z < nz - 1) stage_rows(SG + oZp, m, g, z + 1, y0, TY, tid, nth);
        if (k > 0) {
            stage_rows(SG + oMP, mp, g, z, y0, TY, tid, nth);
            stage_rows(SG + oGQ, gq, g, z, y0, TY, tid, nth);
        }
    }
    cp_async_commit();

    // complex-to-real preprocessing: Z[k] = (X[k] + X*[Hx-k]) + i conj(w^k) (X[k] - X*[Hx-k]).
    // With sum and dif the two brackets and t = conj(w^k) dif, Z[k] = sum + i t and
    // (w^Hx = -1) Z[Hx-k] = sum* + i t*: one item per pair k = 0..Hx/2 loads X[k] and
    // X[Hx-k] once.  The loads of PF items per thread are issued before any is used.
    constexpr int PF = sizeof(V) == 8 ? 8 : 4;
    const int hh = Hx >> 1;
    const int nel = TY * 3 * (hh + 1);
    const long strideK = (long)3 * nz * ny;
    for (int g0 = 0; g0 < nel; g0 += PF * nth) {  // trip count uniform over the CTA (barrier inside)
        const int e0 = g0 + tt;
        V xa[PF], xb[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            const int c = e % 3, rest = e / 3, yl = rest & (TY - 1), kk = rest >> g.lty;
            xa[i] = czero<V>(); xb[i] = czero<V>();
            if (e < nel && y0 + yl < ny) {
                const long base = ((long)z * ny + y0 + yl) * 3 + c;
                xa[i] = ld_nc(P.W + (long)kk * strideK + base);
                xb[i] = ld_nc(P.W + (long)(Hx - kk) * strideK + base);
            }
        }
        if (g0 == 0) {  // the twiddles (first commit group) are needed from here on
            cp_async_wait_group<1>();
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e >= nel) break;
            const int c = e % 3, rest = e / 3, yl = rest & (TY - 1), kk = rest >> g.lty;
            const V Xk = xa[i], Xm = cconj(xb[i]);
            const V sum = cadd(Xk, Xm), dif = csub(Xk, Xm);
            const V t = cmulc(dif, tw[kk]);  // conj(w^k) dif
            V *row = S + (c * TY + yl) * g.rsx;
            V Z;
            Z.x = sum.x - t.y;
            Z.y = sum.y + t.x;
            row[spos<V>(kk)] = Z;
            if (kk != 0 && Hx - kk != kk) {
                Z.x = sum.x + t.y;
                Z.y = t.x - sum.y;
                row[spos<V>(Hx - kk)] = Z;
            }
        }
    }
    __syncthreads();
    {
        const int row = tid / g.Gx, j = tid - row * g.Gx;
        const bool act = row < 3 * TY;
        fft_row<true, false, true, 2, LX>(S + (act ? row : 0) * g.rsx, Hx, g.lhx, j, tw, act);
    }
    cp_async_wait_all();
    if (stg) __syncthreads();

    // local terms
    T he0, he1, he2;
    if (MODE == MODE_MIN) {
        he0 = pick<T>(st->Hext[0], st->Hextf[0], st->Hextw[0]);
        he1 = pick<T>(st->Hext[1], st->Hextf[1], st->Hextw[1]);
        he2 = pick<T>(st->Hext[2], st->Hextf[2], st->Hextw[2]);
    } else {
        he0 = (T)hx0; he1 = (T)hx1; he2 = (T)hx2;
    }
    const T cx = pick<T>(g.cex_x, g.fcex_x, g.wcex[0]), cy = pick<T>(g.cex_y, g.fcex_y, g.wcex[1]),
            cz = pick<T>(g.cex_z, g.fcex_z, g.wcex[2]);
    const T can = pick<T>(g.can, g.fcan, g.wcan);
    const T kfac = (T)0.5 * can;  // 1/(mu0 Ms)
    const T Kuni = pick<T>(g.K, g.fK, g.wK), ux = pick<T>(g.u[0], g.fu[0], g.wu[0]),
            uy = pick<T>(g.u[1], g.fu[1], g.wu[1]), uz = pick<T>(g.u[2], g.fu[2], g.wu[2]);
    const T hs = (T)P.hscale;
    Acc<T> red[NSL];
#pragma unroll
    for (int s = 0; s < NSL; ++s) red[s].zero();

    for (int e = tt; e < TY * nx; e += nth) {
        const int yl = g.fd_nx.div(e), x = e - yl * nx, y = y0 + yl;
        if (y >= ny) continue;
        const long n = ((long)z * ny + y) * nx + x;
        const T d0 = to_field<T>(rel<F>(S + (0 * TY + yl) * g.rsx, x));
        const T d1 = to_field<T>(rel<F>(S + (1 * TY + yl) * g.rsx, x));
        const T d2 = to_field<T>(rel<F>(S + (2 * TY + yl) * g.rsx, x));
        // exchange: sum over present neighbours of (m_j - m_i) / d^2 (free faces)
        T m0, m1, m2, e0 = 0, e1 = 0, e2 = 0;
        if (stg) {
            const int cs = (TY + 2) * nx, ct = TY * nx;    // component strides of the staged rows
            const T *r0 = SG + (yl + 1) * nx + x;          // this cell, component 0
            m0 = r0[0]; m1 = r0[cs]; m2 = r0[2 * cs];
            if (x > 0)      { e0 += cx * (r0[-1] - m0);  e1 += cx * (r0[cs - 1] - m1);  e2 += cx * (r0[2 * cs - 1] - m2); }
            if (x < nx - 1) { e0 += cx * (r0[1] - m0);   e1 += cx * (r0[cs + 1] - m1);  e2 += cx * (r0[2 * cs + 1] - m2); }
            if (y > 0)      { e0 += cy * (r0[-nx] - m0); e1 += cy * (r0[cs - nx] - m1); e2 += cy * (r0[2 * cs - nx] - m2); }
            if (y < ny - 1) { e0 += cy * (r0[nx] - m0);  e1 += cy * (r0[cs + nx] - m1); e2 += cy * (r0[2 * cs + nx] - m2); }
            const T *rz = SG + yl * nx + x;
            if (z > 0)      { const T *q = rz + oZm; e0 += cz * (q[0] - m0); e1 += cz * (q[ct] - m1); e2 += cz * (q[2 * ct] - m2); }
            if (z < nz - 1) { const T *q = rz + oZp; e0 += cz * (q[0] - m0); e1 += cz * (q[ct] - m1); e2 += cz * (q[2 * ct] - m2); }
        } else {
            if constexpr (FROM_T) {
                m0 = ldg(m + n); m1 = ldg(m + N + n); m2 = ldg(m + 2 * N + n);
            } else {
                m0 = from_io<T>(ldg(mio + n)); m1 = from_io<T>(ldg(mio + N + n)); m2 = from_io<T>(ldg(mio + 2 * N + n));
            }
            if (x > 0)      { e0 += cx * (mval(n - 1) - m0);  e1 += cx * (mval(N + n - 1) - m1);  e2 += cx * (mval(2 * N + n - 1) - m2); }
            if (x < nx - 1) { e0 += cx * (mval(n + 1) - m0);  e1 += cx * (mval(N + n + 1) - m1);  e2 += cx * (mval(2 * N + n + 1) - m2); }
            if (y > 0)      { e0 += cy * (mval(n - nx) - m0); e1 += cy * (mval(N + n - nx) - m1); e2 += cy * (mval(2 * N + n - nx) - m2); }
            if (y < ny - 1) { e0 += cy * (mval(n + nx) - m0); e1 += cy * (mval(N + n + nx) - m1); e2 += cy * (mval(2 * N + n + nx) - m2); }
            const long sxy = (long)nx * ny;
            if (z > 0)      { e0 += cz * (mval(n - sxy) - m0); e1 += cz * (mval(N + n - sxy) - m1); e2 += cz * (mval(2 * N + n - sxy) - m2); }
            if (z < nz - 1) { e0 += cz * (mval(n + sxy) - m0); e1 += cz * (mval(N + n + sxy) - m1); e2 += cz * (mval(2 * N + n + sxy) - m2); }
        }
        // uniaxial anisotropy
        const T Kv = P.Kc ? from_io<T>(P.Kc[n]) : Kuni;
        T u0, u1, u2;
        if (P.uc) { u0 = from_io<T>(P.uc[n]); u1 = from_io<T>(P.uc[N + n]); u2 = from_io<T>(P.uc[2 * N + n]); }
        else { u0 = ux; u1 = uy; u2 = uz; }
        const T mu = m0 * u0 + m1 * u1 + m2 * u2;
        const T ka = can * Kv * mu;
        const T H0 = d0 + e0 + ka * u0 + he0;
        const T H1 = d1 + e1 + ka * u1 + he1;
        const T H2 = d2 + e2 + ka * u2 + he2;
        if (MODE == MODE_HEFF) {
            P.H_out[n] = to_io(hs * H0); P.H_out[N + n] = to_io(hs * H1); P.H_out[2 * N + n] = to_io(hs * H2);
            continue;
        }
        red[SL_MX].add(m0); red[SL_MY].add(m1); red[SL_MZ].add(m2);
        const T mhe = m0 * he0 + m1 * he1 + m2 * he2;
        if (MODE == MODE_ENERGY) {
            if constexpr (sizeof(T) == 4) {
                // float path: every per-cell product enters its sum exactly
                red[SL_ED].add_prod(m0, d0); red[SL_ED].add_prod(m1, d1); red[SL_ED].add_prod(m2, d2);
                red[SL_EEX].add_prod(m0, e0); red[SL_EEX].add_prod(m1, e1); red[SL_EEX].add_prod(m2, e2);
                red[SL_EAN].add_prod(Kv, (T)1 - mu * mu);
                red[SL_EZ].add_prod(m0, he0); red[SL_EZ].add_prod(m1, he1); red[SL_EZ].add_prod(m2, he2);
            } else {
                red[SL_ED].add(m0 * d0 + m1 * d1 + m2 * d2);
                red[SL_EEX].add(m0 * e0 + m1 * e1 + m2 * e2);
                red[SL_EAN].add(Kv * ((T)1 - mu * mu));
                red[SL_EZ].add(mhe);
            }
            continue;
        }
        // projected gradient g = m x (m x H) = (m.H) m - |m|^2 H (the triple
        // product identity; orthogonal to m for any |m|, which keeps the
        // midpoint step norm-preserving even as rounding moves |m| off 1)
        const T mh = m0 * H0 + m1 * H1 + m2 * H2;
        const T mm = m0 * m0 + m1 * m1 + m2 * m2;
        const T g0 = mh * m0 - mm * H0, g1 = mh * m1 - mm * H1, g2 = mh * m2 - mm * H2;
        red[SL_T2].maxv(g0 * g0 + g1 * g1 + g2 * g2);  // |m x H|^2 = |g|^2 for |m| = 1
        // energy density / (mu0 Ms V): -m.H/2 - m.H_ext/2 + K/(mu0 Ms)
        if constexpr (sizeof(T) == 4) {
            const T h0 = (T)-0.5 * m0, h1 = (T)-0.5 * m1, h2 = (T)-0.5 * m2;  // exact halvings
            red[SL_ET].add_prod(h0, H0); red[SL_ET].add_prod(h1, H1); red[SL_ET].add_prod(h2, H2);
            red[SL_ET].add_prod(h0, he0); red[SL_ET].add_prod(h1, he1); red[SL_ET].add_prod(h2, he2);
            red[SL_ET].add_prod(kfac, Kv);
        } else {
            red[SL_ET].add((T)-0.5 * (mh + mhe) + kfac * Kv);
        }
        T *gout = (k & 1) ? P.gbuf[1] : P.gbuf[0];
        if (k > 0) {
            T p0, p1, p2, q0, q1, q2;
            if (stg) {
                const int sn = yl * nx + x, ct = TY * nx;
                p0 = SG[oMP + sn]; p1 = SG[oMP + ct + sn]; p2 = SG[oMP + 2 * ct + sn];
                q0 = SG[oGQ + sn]; q1 = SG[oGQ + ct + sn]; q2 = SG[oGQ + 2 * ct + sn];
            } else {
                p0 = mp[n]; p1 = mp[N + n]; p2 = mp[2 * N + n];
                q0 = gq[n]; q1 = gq[N + n]; q2 = gq[2 * N + n];
            }
            const T s0 = m0 - p0, s1 = m1 - p1, s2 = m2 - p2;
            const T y0v = g0 - q0, y1v = g1 - q1, y2v = g2 - q2;
            if constexpr (sizeof(T) == 4) {
                // float path: exact products, compensated sums (the step size
                // needs s.y, a difference of nearly equal sums near convergence)
                red[SL_SS].add_prod(s0, s0); red[SL_SS].add_prod(s1, s1); red[SL_SS].add_prod(s2, s2);
                red[SL_SY].add_prod(s0, y0v); red[SL_SY].add_prod(s1, y1v); red[SL_SY].add_prod(s2, y2v);
                red[SL_YY].add_prod(y0v, y0v); red[SL_YY].add_prod(y1v, y1v); red[SL_YY].add_prod(y2v, y2v);
            } else {
                red[SL_SS].add(s0 * s0 + s1 * s1 + s2 * s2);
                red[SL_SY].add(s0 * y0v + s1 * y1v + s2 * y2v);
                red[SL_YY].add(y0v * y0v + y1v * y1v + y2v * y2v);
            }
        }
        gout[n] = g0; gout[N + n] = g1; gout[2 * N + n] = g2;
    }
    if (MODE == MODE_HEFF) return;

    // CTA reduction: the FFT rows are done with; stage every thread's
    // accumulators in shared memory and let warp s reduce slot s.
    __syncthreads();
    Acc<T> *stage = reinterpret_cast<Acc<T> *>(smem_raw);
    if (tid < nth) {
#pragma unroll
        for (int s = 0; s < NSL; ++s) stage[s * nth + tid] = red[s];
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int s = (tid < nth ? warp : NSL); s < NSL; s += nth >> 5) {  // warp w reduces slots w, w + nwarps, ...
        const bool isMax = (MODE == MODE_MIN && s == SL_T2);
        Acc<T> a = stage[s * nth + lane];
        for (int i = lane + 32; i < nth; i += 32) {
            if (isMax) a.maxv(stage[s * nth + i]); else a.add(stage[s * nth + i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const Acc<T> b = a.shfl_down(o);
            if (isMax) a.maxv(b); else a.add(b);
        }
        if (lane == 0) P.partials[(long)bid * RED_NSLOT + s] = a.value();
    }
    // the last CTA to arrive finishes the evaluation
    __shared__ int s_last;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = (atomicAdd(P.counter, 1u) == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (s_last && warp == 0) {   // no early return: a persistent batch CTA goes on to its next work item
        __threadfence();
        finish_iteration<MODE>(g, P.partials, nblk, st, h, use_cond, g.nbody);
        if (lane == 0) *P.counter = 0u;
    }
}

template <typename T, typename F, int MODE, int LX>
__global__ void __launch_bounds__(768) k_xinv(Geom g, FieldPtrs<T, F> P, double hx0, double hx1, double hx2,
                                              cudaGraphConditionalHandle h, int use_cond)
{
    xinv_body<T, F, MODE, LX>(g, P, hx0, hx1, hx2, h, use_cond, threadIdx.x, blockDim.x, blockIdx.x, blockIdx.y,
                           blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// launch shapes and buffers of a problem's field kernels
// ---------------------------------------------------------------------------
template <typename T, typename F = T> FieldPtrs<T, F> make_ptrs(mm_problem *p)
{
    typedef typename cvec<F>::type V;
    FieldPtrs<T, F> P;
    P.m_src = nullptr; P.H_out = nullptr;
    P.mbuf[0] = (T *)p->mbuf[0]; P.mbuf[1] = (T *)p->mbuf[1];
    P.gbuf[0] = (T *)p->gbuf[0]; P.gbuf[1] = (T *)p->gbuf[1];
    P.W = (V *)p->W; P.W2 = (V *)p->W2; P.Nhat = (const F *)p->Nhat;
    P.tw_px = (const V *)p->tw_px; P.tw_py = (const V *)p->tw_py; P.tw_pz = (const V *)p->tw_pz;
    typedef typename io_of<T>::type IO;
    P.Kc = (const IO *)p->Kc; P.uc = (const IO *)p->uc;
    P.partials = p->partials; P.st = p->st; P.counter = p->counter;
    P.hscale = 1.0;
    return P;
}

static inline int round32(int n) { return (n + 31) & ~31; }
template <typename T> int threads_x(const Geom &g) { return round32(3 * g.TY * g.Gx); }
template <typename T> int threads_xf(const Geom &g) { return round32(3 * g.TYF * g.Gx); }
template <typename T> size_t smem_xf_t(const Geom &g)
{
    typedef typename cvec<T>::type V;
    return (size_t)3 * g.TYF * g.rsx * sizeof(V) + (size_t)g.Px * sizeof(V);
}
template <typename T> int threads_yz(const Geom &g) { return round32(g.RB * g.Gy); }

template <typename T> size_t smem_x_t(const Geom &g)
{
    typedef typename cvec<T>::type V;
    size_t rows = (size_t)3 * g.TY * g.rsx * sizeof(V) + (size_t)g.Px * sizeof(V);
    if (sizeof(T) == 4 && g.stage) rows = stage_offset<T>(g) + (size_t)(15 * g.TY + 6) * g.nx * sizeof(T);
    const size_t stage = (size_t)NSL * threads_x<T>(g) * sizeof(Acc<T>);
    return rows > stage ? rows : stage;
}
template <typename T> size_t smem_yz_t(const Geom &g)
{
    typedef typename cvec<T>::type V;
    // the float kernel also holds the Py twiddles (the double kernel reads them from global memory)
    return (size_t)3 * g.nz * g.rsy * sizeof(V) + (sizeof(T) == 4 ? (size_t)g.Py * sizeof(V) : 0);
}

// The field kernels are compiled for FFT row lengths 2^6 .. 2^10 (template
// parameter LX of the x kernels: log2 Hx; LY of the y-z kernel: log2 Py) and
// once for any length (0); these launchers pick the instance.
__host__ __device__ inline int lc_of(int logL) { return MM_FFT_SPECIALISED(logL) ? logL : 0; }
#define MM_LC_CASES(X) X(0) X(6) X(7) X(8) X(9) X(10)
// Double-word (F = dfloat) kernels are compiled for the lengths 512 and 1024
// only (rows of films 257 .. 1024 cells long, and 129 .. 512 wide), other
// lengths take the generic code: their unrolled double-word arithmetic makes
// every compiled length expensive to build.
template <typename F> constexpr bool lc_compiled(int L) { return true; }
template <> constexpr bool lc_compiled<dfloat>(int L) { return L == 0 || L == 9 || L == 10; }
template <typename F> __host__ __device__ inline int lc_of_f(int logL)
{
    const int L = lc_of(logL);
    return lc_compiled<F>(L) ? L : 0;
}

} // namespace
