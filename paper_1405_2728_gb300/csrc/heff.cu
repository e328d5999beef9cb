// Effective-field and minimiser-step kernels (sm_103a).
//
// One evaluation of H_eff (Eq. effective_field; Sections 3 and 4) is three
// kernels over the zero-padded grid for films (bulk grids replace k_yz by
// the three passes of bulk.cu); in the minimiser (Section 2) the last of
// them also finishes the iteration:
//
//  k_xfwd     per (z, tile of TYF rows): optional minimiser step (the closed
//             form of the midpoint scheme, Eq. implicit_gradient_descent, or
//             the renormalised explicit step) fused with the real-to-complex
//             FFT along x of the three components, zero padding nx -> Px,
//             written transposed to the spectrum W[kx][z][y][c].
//  k_yz       per x-frequency kx: FFT along y (padding ny -> Py) in shared
//             memory; then per ky, in registers, the z direction as a direct
//             convolution with the tensor transformed along x and y
//             (H^ = -Ms N m^, nz <= 4, normalisation folded into the tensor);
//             then the inverse FFT along y keeping the first ny rows.
//  k_xinv     per (z, tile of TY rows): complex-to-real inverse FFT along x keeping nx
//             values, then the local terms: exchange (six-point stencil, free
//             faces), uniaxial anisotropy, Zeeman.  Depending on the mode it
//             writes H, or accumulates the energy terms, or forms the projected
//             gradient g = m x (m x H) (Eq. projected_direction) with the
//             Barzilai-Borwein sums s.s, s.y, y.y (Eq. stepsize), max |m x H|,
//             the energy and sum m.  Each CTA stores its partial sums; the last
//             CTA to finish sums them in a fixed order (deterministic), picks
//             the step size tau^1 / tau^2 alternately (Eq. stepsize), applies
//             the stop rule and sets the device-side loop condition.
//
// Sums are accumulated in double on the double path.  On the float path each
// per-cell product enters its sum exactly (TwoProduct with one FMA) and the
// sums are compensated float pairs (TwoSum, Knuth), about 46 significant
// bits; partial sums are always combined across CTAs in double.
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "fft.cuh"

namespace {

template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

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
                                           int nrows)
{
    constexpr int CH = 16 / sizeof(T);
    const int nx = g.nx, nc = g.fd_nc.d;
    const int tot = 3 * nrows * nc;
    const long plane = (long)z * g.ny * nx;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
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
template <typename T, bool MIN, int LX>
__global__ void __launch_bounds__(768) k_xfwd(Geom g, FieldPtrs<T> P)
{
    typedef typename cvec<T>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int TY = g.TYF, y0 = blockIdx.x * TY, z = blockIdx.y;
    const int nx = g.nx, ny = g.ny, Px = g.Px;
    const long N = g.N;
    V *tw = S + 3 * TY * g.rsx;  // Px twiddles exp(-2 pi i t / Px)
    load_twiddles(tw, P.tw_px, Px);

    const T *src;
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
            tau = pick<T>(st->tau, st->tauf);
            step_kind = st->step_kind;
        } else {
            src = cur ? P.mbuf[1] : P.mbuf[0];
        }
    } else {
        src = P.m_src;
    }
    // load (and step) the tile; row (c, yl) holds Px reals
#pragma unroll(sizeof(T) == 4 ? 2 : 1)
    for (int e = tid; e < TY * nx; e += nth) {
        const int yl = g.fd_nx.div(e), x = e - yl * nx, y = y0 + yl;
        T m0 = 0, m1 = 0, m2 = 0;
        if (y < ny) {
            const long n = ((long)z * ny + y) * nx + x;
            m0 = __ldg(src + n); m1 = __ldg(src + N + n); m2 = __ldg(src + 2 * N + n);
            if (MIN && dst) {
                const T g0 = __ldg(gp + n), g1 = __ldg(gp + N + n), g2 = __ldg(gp + 2 * N + n);
                if (step_kind == MM_STEP_CAYLEY) {
                    const T q = (T)0.25 * tau * tau * (g0 * g0 + g1 * g1 + g2 * g2);
                    const T a = (T)1 - q, inv = (T)1 / ((T)1 + q);
                    m0 = (a * m0 - tau * g0) * inv;
                    m1 = (a * m1 - tau * g1) * inv;
                    m2 = (a * m2 - tau * g2) * inv;
                    if (sizeof(T) == 4) {
                        // float path only: the closed form keeps |m| = 1 exactly in
                        // exact arithmetic; in float its rounding drifts ~1e-7 per
                        // step, so the float path renormalises (the double path keeps
                        // the pure midpoint form, drift ~1e-16 per step)
                        const T r = rsqrtf((float)(m0 * m0 + m1 * m1 + m2 * m2));
                        m0 *= r; m1 *= r; m2 *= r;
                    }
                } else {
                    m0 -= tau * g0; m1 -= tau * g1; m2 -= tau * g2;
                    const T inv = (T)1 / sqrt(m0 * m0 + m1 * m1 + m2 * m2);
                    m0 *= inv; m1 *= inv; m2 *= inv;
                }
                dst[n] = m0; dst[N + n] = m1; dst[2 * N + n] = m2;
            }
        }
        rel<T>(S + (0 * TY + yl) * g.rsx, x) = m0;
        rel<T>(S + (1 * TY + yl) * g.rsx, x) = m1;
        rel<T>(S + (2 * TY + yl) * g.rsx, x) = m2;
    }
    const int npad = Px - nx;
    for (int e = tid; e < 3 * TY * npad; e += nth) {
        const int row = g.fd_padx.div(e), x = nx + (e - row * npad);
        rel<T>(S + row * g.rsx, x) = 0;
    }
    __syncthreads();

    // complex FFT of length Hx of the packed rows (upper half zero)
    {
        const int row = tid / g.Gx, j = tid - row * g.Gx;
        const bool act = row < 3 * TY;
        fft_row<false, true, false, 2, LX>(S + (act ? row : 0) * g.rsx, g.Hx, g.lhx, j, tw, act);
    }

    // unpack to the real-input spectrum X[k], k = 0..Hx, and store transposed
    const int Hx = g.Hx, C = g.C;
    for (int e = tid; e < TY * 3 * C; e += nth) {
        const int c = e % 3, rest = e / 3, yl = rest & (TY - 1), k = rest >> g.ltyf;
        const int y = y0 + yl;
        const V *row = S + (c * TY + yl) * g.rsx;
        const V Zk = row[spos<V>(k == Hx ? 0 : k)];
        const V Zm = cconj(row[spos<V>(k == 0 ? 0 : Hx - k)]);
        const V w = tw[k];
        const V sum = cadd(Zk, Zm), dif = csub(Zk, Zm);
        // X = (sum - i w dif) / 2
        const V wd = cmul(w, dif);
        V X;
        X.x = (T)0.5 * (sum.x + wd.y);
        X.y = (T)0.5 * (sum.y - wd.x);
        if (y < ny) P.W[(((long)k * g.nz + z) * ny + y) * 3 + c] = X;
    }
}

// ---------------------------------------------------------------------------
// k_yz
// ---------------------------------------------------------------------------
// the double kernel runs fewer, fatter threads (its z-phase keeps ~100
// doubles live); the y rows are then transformed in batches of RB rows
template <typename T> struct YZBound { static constexpr int v = sizeof(T) == 8 ? 512 : 768; };

template <typename T, int PZ, int LY>
__global__ void __launch_bounds__(YZBound<T>::v) k_yz(Geom g, FieldPtrs<T> P)
{
    typedef typename cvec<T>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int kx = blockIdx.x;
    const int ny = g.ny, nz = g.nz, Py = g.Py;
    const int nrow = 3 * nz;
    V *Wk = P.W + (long)kx * nrow * ny;
    // Py twiddles: a shared copy in float; the double kernel reads them from
    // global memory (L1), which keeps its shared memory within two CTAs per SM
    const V *tw;
    if constexpr (sizeof(T) == 4) {
        V *tws = S + nrow * g.rsy;
        load_twiddles_async(tws, P.tw_py, Py);
        tw = tws;
    } else {
        tw = P.tw_py;
    }

    // Wk[z][y][c] -> row (c, z); PF loads per thread in flight before use
    constexpr int PF = sizeof(T) == 4 ? 8 : 4;
    const int tot = nrow * ny;
    for (int e0 = tid; e0 < tot; e0 += PF * nth) {
        V v[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e < tot) v[i] = __ldcg(Wk + e);
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
    for (int e = tid; e < nrow * npad; e += nth) {
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
    const T *Kk = P.Nhat + (long)kx * NZM * 6 * kst;
    for (int ky = tid; ky < Py; ky += nth) {
        const int pky = spos<V>(ky);
        const int kyr = ky <= hy ? ky : Py - ky;
        const T sy = ky <= hy ? (T)1 : (T)-1;
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
            const T *kd = Kk + (long)dz * 6 * kst + kyr;
            const T kxx = ldg(kd), kyy = ldg(kd + kst), kzz = ldg(kd + 2 * kst);
            const T kxy = sy * ldg(kd + 3 * kst), kxz = ldg(kd + 4 * kst), kyz = sy * ldg(kd + 5 * kst);
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
                        const T sxz = side ? -kxz : kxz, syz = side ? -kyz : kyz;
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

    for (int e = tid; e < nrow * ny; e += nth) {
        const int c = e % 3, rest = e / 3, zz = g.fd_ny.div(rest), y = rest - zz * ny;
        Wk[e] = S[(c * nz + zz) * g.rsy + spos<V>(y)];
    }
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
    double tot[NSL];
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
        const bool isMax = (MODE == MODE_MIN && s == SL_T2);
        double v = 0.0;
        for (int b = lane; b < nblk; b += 32) {
            const double x = __ldcg(partials + (long)b * RED_NSLOT + s);
            v = isMax ? fmax(v, x) : v + x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, v, o);
            v = isMax ? fmax(v, y) : v + y;
        }
        tot[s] = v;
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
        st->k = k + 1;
        stop = 0;
    }
    if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// k_xinv
// ---------------------------------------------------------------------------
template <typename T, int MODE, int LX>
__global__ void __launch_bounds__(768) k_xinv(Geom g, FieldPtrs<T> P, double hx0, double hx1, double hx2,
                                              cudaGraphConditionalHandle h, int use_cond)
{
    typedef typename cvec<T>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int TY = g.TY, y0 = blockIdx.x * TY, z = blockIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz, Hx = g.Hx;
    const long N = g.N;
    V *tw = S + 3 * TY * g.rsx;

    MinState *st = P.st;
    long k = 0;
    int cur = 0;
    const T *m;
    const T *mp = nullptr, *gq = nullptr;
    if (MODE == MODE_MIN) {
        k = st->k;
        cur = st->base ^ (int)(k & 1);
        m = cur ? P.mbuf[1] : P.mbuf[0];
        mp = cur ? P.mbuf[0] : P.mbuf[1];
        gq = (k & 1) ? P.gbuf[0] : P.gbuf[1];  // g_{k-1}
    } else {
        m = P.m_src;
    }
    // the float kernel stages the local terms' inputs -- m on planes z-1, z,
    // z+1 (rows y0-1 .. y0+TY on its own plane), m_{k-1} and g_{k-1} -- with
    // cp.async now; they arrive while the inverse x-FFT runs
    const bool stg = sizeof(T) == 4 && MODE == MODE_MIN && g.stage;
    T *SG = reinterpret_cast<T *>(smem_raw + stage_offset<T>(g));
    const int oZm = 3 * (TY + 2) * nx, oZp = oZm + 3 * TY * nx, oMP = oZp + 3 * TY * nx, oGQ = oMP + 3 * TY * nx;
    load_twiddles_async(tw, P.tw_px, g.Px);
    cp_async_commit();
    if (stg) {
        stage_rows(SG, m, g, z, y0 - 1, TY + 2);
        if (z > 0) stage_rows(SG + oZm, m, g, z - 1, y0, TY);
        if (z < nz - 1) stage_rows(SG + oZp, m, g, z + 1, y0, TY);
        if (k > 0) {
            stage_rows(SG + oMP, mp, g, z, y0, TY);
            stage_rows(SG + oGQ, gq, g, z, y0, TY);
        }
    }
    cp_async_commit();

    // complex-to-real preprocessing: Z[k] = (X[k] + X*[Hx-k]) + i conj(w^k) (X[k] - X*[Hx-k]);
    // the spectrum loads of PF elements per thread are issued before any is used
    constexpr int PF = sizeof(T) == 4 ? 8 : 4;
    const int nel = TY * 3 * Hx;
    const long strideK = (long)3 * nz * ny;
    for (int g0 = 0; g0 < nel; g0 += PF * nth) {  // trip count uniform over the CTA (barrier inside)
        const int e0 = g0 + tid;
        V xa[PF], xb[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            const int c = e % 3, rest = e / 3, yl = rest & (TY - 1), kk = rest >> g.lty;
            xa[i] = czero<V>(); xb[i] = czero<V>();
            if (e < nel && y0 + yl < ny) {
                const long base = ((long)z * ny + y0 + yl) * 3 + c;
                xa[i] = __ldg(P.W + (long)kk * strideK + base);
                xb[i] = __ldg(P.W + (long)(Hx - kk) * strideK + base);
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
            V Z;
            Z.x = sum.x - t.y;
            Z.y = sum.y + t.x;
            S[(c * TY + yl) * g.rsx + spos<V>(kk)] = Z;
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
        he0 = pick<T>(st->Hext[0], st->Hextf[0]);
        he1 = pick<T>(st->Hext[1], st->Hextf[1]);
        he2 = pick<T>(st->Hext[2], st->Hextf[2]);
    } else {
        he0 = (T)hx0; he1 = (T)hx1; he2 = (T)hx2;
    }
    const T cx = pick<T>(g.cex_x, g.fcex_x), cy = pick<T>(g.cex_y, g.fcex_y), cz = pick<T>(g.cex_z, g.fcex_z);
    const T can = pick<T>(g.can, g.fcan);
    const T kfac = (T)0.5 * can;  // 1/(mu0 Ms)
    const T Kuni = pick<T>(g.K, g.fK), ux = pick<T>(g.u[0], g.fu[0]), uy = pick<T>(g.u[1], g.fu[1]),
            uz = pick<T>(g.u[2], g.fu[2]);
    const T hs = (T)P.hscale;
    Acc<T> red[NSL];
#pragma unroll
    for (int s = 0; s < NSL; ++s) red[s].zero();

    for (int e = tid; e < TY * nx; e += nth) {
        const int yl = g.fd_nx.div(e), x = e - yl * nx, y = y0 + yl;
        if (y >= ny) continue;
        const long n = ((long)z * ny + y) * nx + x;
        const T d0 = rel<T>(S + (0 * TY + yl) * g.rsx, x);
        const T d1 = rel<T>(S + (1 * TY + yl) * g.rsx, x);
        const T d2 = rel<T>(S + (2 * TY + yl) * g.rsx, x);
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
            m0 = __ldg(m + n); m1 = __ldg(m + N + n); m2 = __ldg(m + 2 * N + n);
            if (x > 0)      { e0 += cx * (m[n - 1] - m0);  e1 += cx * (m[N + n - 1] - m1);  e2 += cx * (m[2 * N + n - 1] - m2); }
            if (x < nx - 1) { e0 += cx * (m[n + 1] - m0);  e1 += cx * (m[N + n + 1] - m1);  e2 += cx * (m[2 * N + n + 1] - m2); }
            if (y > 0)      { e0 += cy * (m[n - nx] - m0); e1 += cy * (m[N + n - nx] - m1); e2 += cy * (m[2 * N + n - nx] - m2); }
            if (y < ny - 1) { e0 += cy * (m[n + nx] - m0); e1 += cy * (m[N + n + nx] - m1); e2 += cy * (m[2 * N + n + nx] - m2); }
            const long sxy = (long)nx * ny;
            if (z > 0)      { e0 += cz * (m[n - sxy] - m0); e1 += cz * (m[N + n - sxy] - m1); e2 += cz * (m[2 * N + n - sxy] - m2); }
            if (z < nz - 1) { e0 += cz * (m[n + sxy] - m0); e1 += cz * (m[N + n + sxy] - m1); e2 += cz * (m[2 * N + n + sxy] - m2); }
        }
        // uniaxial anisotropy
        const T Kv = P.Kc ? P.Kc[n] : Kuni;
        T u0, u1, u2;
        if (P.uc) { u0 = P.uc[n]; u1 = P.uc[N + n]; u2 = P.uc[2 * N + n]; }
        else { u0 = ux; u1 = uy; u2 = uz; }
        const T mu = m0 * u0 + m1 * u1 + m2 * u2;
        const T ka = can * Kv * mu;
        const T H0 = d0 + e0 + ka * u0 + he0;
        const T H1 = d1 + e1 + ka * u1 + he1;
        const T H2 = d2 + e2 + ka * u2 + he2;
        if (MODE == MODE_HEFF) {
            P.H_out[n] = hs * H0; P.H_out[N + n] = hs * H1; P.H_out[2 * N + n] = hs * H2;
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
#pragma unroll
    for (int s = 0; s < NSL; ++s) stage[s * nth + tid] = red[s];
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    for (int s = warp; s < NSL; s += nth >> 5) {  // warp w reduces slots w, w + nwarps, ...
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
        const unsigned nblk = gridDim.x * gridDim.y;
        s_last = (atomicAdd(P.counter, 1u) == nblk - 1);
    }
    __syncthreads();
    if (!s_last || warp != 0) return;
    __threadfence();
    finish_iteration<MODE>(g, P.partials, gridDim.x * gridDim.y, st, h, use_cond, g.nbody);
    if (lane == 0) *P.counter = 0u;
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__global__ void k_init_state(MinState *st, double tau0, double tol_abs, double h0, double h1, double h2,
                             long max_iter, int step_kind, unsigned long long timeout_ns, int reset_base,
                             int tau_rule, double kappa)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (reset_base) st->base = 0;
    else st->base = st->base ^ (int)(st->k & 1);   // continue from the previous result
    st->tau0 = tau0; st->tol_abs = tol_abs;
    st->Hext[0] = h0; st->Hext[1] = h1; st->Hext[2] = h2;
    st->Hextf[0] = (float)h0; st->Hextf[1] = (float)h1; st->Hextf[2] = (float)h2;
    st->max_iter = max_iter; st->step_kind = step_kind;
    st->tau_rule = tau_rule; st->kappa = kappa;
    st->timeout_ns = timeout_ns; st->t_start_ns = 0;
    st->k = 0; st->tau = tau0; st->tauf = (float)tau0; st->status = MMS_RUNNING; st->evals = 0; st->launches = 1;
    st->max_torque = 0;
}

__global__ void k_record(const MinState *st, StepRecord *rec, int step)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    StepRecord r;
    r.mavg[0] = st->mavg[0]; r.mavg[1] = st->mavg[1]; r.mavg[2] = st->mavg[2];
    r.max_torque = st->max_torque; r.energy = st->energy[4];
    r.iters = st->k; r.evals = st->evals; r.launches = st->launches + 1; r.status = st->status;
    rec[step] = r;
}

template <typename T>
__global__ void k_copy_result(const MinState *st, const T *b0, const T *b1, T *dst, long n3)
{
    const T *src = (st->base ^ (int)(st->k & 1)) ? b1 : b0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n3; i += (long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

template <typename T>
__global__ void k_twiddle(typename cvec<T>::type *tw, int L)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)L, &s, &c);
    typename cvec<T>::type w;
    w.x = (T)c; w.y = (T)(-s);
    tw[t] = w;
}

template <typename T>
__global__ void k_convert(T *dst, const double *src, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
template <typename T> FieldPtrs<T> make_ptrs(mm_problem *p)
{
    typedef typename cvec<T>::type V;
    FieldPtrs<T> P;
    P.m_src = nullptr; P.H_out = nullptr;
    P.mbuf[0] = (T *)p->mbuf[0]; P.mbuf[1] = (T *)p->mbuf[1];
    P.gbuf[0] = (T *)p->gbuf[0]; P.gbuf[1] = (T *)p->gbuf[1];
    P.W = (V *)p->W; P.W2 = (V *)p->W2; P.Nhat = (const T *)p->Nhat;
    P.tw_px = (const V *)p->tw_px; P.tw_py = (const V *)p->tw_py; P.tw_pz = (const V *)p->tw_pz;
    P.Kc = (const T *)p->Kc; P.uc = (const T *)p->uc;
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
inline int lc_of(int logL) { return MM_FFT_SPECIALISED(logL) ? logL : 0; }
#define MM_LC_CASES(X) X(0) X(6) X(7) X(8) X(9) X(10)

template <typename T, bool MIN>
cudaError_t launch_xfwd(const Geom &g, const FieldPtrs<T> &P, cudaStream_t s)
{
    const dim3 grid((g.ny + g.TYF - 1) / g.TYF, g.nz);
    const int thr = threads_xf<T>(g);
    const size_t sm = smem_xf_t<T>(g);
    switch (lc_of(g.lhx)) {
#define C(L) case L: k_xfwd<T, MIN, L><<<grid, thr, sm, s>>>(g, P); break;
        MM_LC_CASES(C)
#undef C
    }
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_xinv(const Geom &g, const FieldPtrs<T> &P, cudaStream_t s, const double *hext,
                        cudaGraphConditionalHandle h, int use_cond)
{
    const dim3 grid((g.ny + g.TY - 1) / g.TY, g.nz);
    const int thr = threads_x<T>(g);
    const size_t sm = smem_x_t<T>(g);
    const double h0 = hext ? hext[0] : 0.0, h1 = hext ? hext[1] : 0.0, h2 = hext ? hext[2] : 0.0;
    switch (lc_of(g.lhx)) {
#define C(L) case L: k_xinv<T, MODE, L><<<grid, thr, sm, s>>>(g, P, h0, h1, h2, h, use_cond); break;
        MM_LC_CASES(C)
#undef C
    }
    return cudaGetLastError();
}

template <typename T, int PZ>
cudaError_t launch_yz(const Geom &g, const FieldPtrs<T> &P, cudaStream_t s)
{
    switch (lc_of(g.lpy)) {
#define C(L) case L: k_yz<T, PZ, L><<<g.C, threads_yz<T>(g), smem_yz_t<T>(g), s>>>(g, P); break;
        MM_LC_CASES(C)
#undef C
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_yz_any(const Geom &g, const FieldPtrs<T> &P, cudaStream_t s)
{
    switch (g.Pz) {
    case 1: return launch_yz<T, 1>(g, P, s);
    case 4: return launch_yz<T, 4>(g, P, s);
    case 8: return launch_yz<T, 8>(g, P, s);
    default: return cudaErrorInvalidValue;  // Pz = 2 does not occur (nz = 1 gives 1, nz = 2 gives 4)
    }
}

// the y-z stage: the film kernel, or the three passes of the bulk layout
template <typename T>
cudaError_t launch_conv(const Geom &g, const FieldPtrs<T> &P, cudaStream_t s)
{
    return g.bulk ? mm_bulk_conv(g, P, s, -1) : launch_yz_any<T>(g, P, s);
}

template <typename F> cudaError_t smem_attr(F *f, size_t bytes)
{
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// dynamic shared memory limits of the instances this geometry launches
template <typename T> cudaError_t configure_t(const Geom &g, size_t sxf, size_t sx, size_t syz)
{
    cudaError_t e = cudaSuccess;
    switch (lc_of(g.lhx)) {
#define C(L)                                                                                     \
    case L:                                                                                      \
        if ((e = smem_attr(k_xfwd<T, false, L>, sxf)) || (e = smem_attr(k_xfwd<T, true, L>, sxf)) || \
            (e = smem_attr(k_xinv<T, MODE_HEFF, L>, sx)) || (e = smem_attr(k_xinv<T, MODE_ENERGY, L>, sx)) || \
            (e = smem_attr(k_xinv<T, MODE_MIN, L>, sx)))                                         \
            return e;                                                                            \
        break;
        MM_LC_CASES(C)
#undef C
    }
    if (g.bulk) return cudaSuccess;
    switch (lc_of(g.lpy)) {
#define C(L)                                                                                     \
    case L:                                                                                      \
        if (g.Pz == 1) return smem_attr(k_yz<T, 1, L>, syz);                                     \
        if (g.Pz == 4) return smem_attr(k_yz<T, 4, L>, syz);                                     \
        if (g.Pz == 8) return smem_attr(k_yz<T, 8, L>, syz);                                     \
        return cudaErrorInvalidValue;
        MM_LC_CASES(C)
#undef C
    }
    return cudaErrorInvalidValue;
}

// Launch-shape autotuner: time every admissible rows-per-tile of the
// x-forward kernel and, separately, of the x-inverse kernel (the two are
// independent: the spectrum layout does not depend on the tile), and every
// rows-per-batch RB of the y-z kernel, on this problem's own buffers (three
// repetitions, best taken); keep the fastest of each.  The kernels run in
// their minimiser modes on the zeroed state of a fresh problem.
template <typename T> cudaError_t autotune_t(mm_problem *p, const int *tys, int nty, const int *rbs, int nrb,
                                             cudaStream_t s)
{
    Geom g = p->g;
    FieldPtrs<T> P = make_ptrs<T>(p);
    P.m_src = (const T *)p->mbuf[0];
    P.H_out = (T *)p->gbuf[0];
    cudaEvent_t a, b;
    cudaError_t e;
    // a minimiser state past its first iteration, so that the step and the
    // step-size sums are part of what is timed (the zeroed buffers make it
    // arithmetic on zeros and NaNs, which costs the same)
    MinState ms;
    memset(&ms, 0, sizeof ms);
    ms.k = 1;
    ms.tau = ms.tau0 = 1e-9;
    ms.tauf = 1e-9f;
    ms.max_iter = 1L << 40;
    ms.status = MMS_RUNNING;
    if ((e = cudaMemcpyAsync(p->st, &ms, sizeof ms, cudaMemcpyHostToDevice, s)) || (e = cudaStreamSynchronize(s)))
        return e;
    if ((e = cudaEventCreate(&a))) return e;
    if ((e = cudaEventCreate(&b))) { cudaEventDestroy(a); return e; }
    for (int which = 0; which < 2 && !e; ++which) {
        float best = 1e30f;
        int bty = tys[0];
        for (int i = 0; i < nty && !e; ++i) {
            if (which == 0) { g.TYF = tys[i]; g.ltyf = mm_ilog2(g.TYF); }
            else { g.TY = tys[i]; g.lty = mm_ilog2(g.TY); }
            float tmin = 1e30f;
            for (int r = 0; r < 3 && !e; ++r) {
                cudaEventRecord(a, s);
                if (which == 0) launch_xfwd<T, true>(g, P, s);
                else launch_xinv<T, MODE_MIN>(g, P, s, nullptr, 0, 0);
                cudaEventRecord(b, s);
                if ((e = cudaGetLastError()) || (e = cudaEventSynchronize(b))) break;
                float t = 0;
                cudaEventElapsedTime(&t, a, b);
                if (t < tmin) tmin = t;
            }
            if (tmin < best) { best = tmin; bty = tys[i]; }
        }
        if (which == 0) { g.TYF = bty; g.ltyf = mm_ilog2(bty); }
        else { g.TY = bty; g.lty = mm_ilog2(bty); }
    }
    float best = 1e30f;
    int brb = rbs[0];
    for (int i = 0; i < nrb && !e && !g.bulk; ++i) {
        g.RB = rbs[i];
        float tmin = 1e30f;
        for (int r = 0; r < 3 && !e; ++r) {
            cudaEventRecord(a, s);
            e = launch_yz_any<T>(g, P, s);
            cudaEventRecord(b, s);
            if (e || (e = cudaEventSynchronize(b))) break;
            float t = 0;
            cudaEventElapsedTime(&t, a, b);
            if (t < tmin) tmin = t;
        }
        if (tmin < best) { best = tmin; brb = rbs[i]; }
    }
    g.RB = brb;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!e) e = cudaMemsetAsync(p->st, 0, sizeof(MinState), s);
    if (!e) e = cudaMemsetAsync(p->counter, 0, 64, s);
    if (!e) p->g = g;
    return e;
}

// Field chain for MODE_HEFF / MODE_ENERGY on caller-provided m (and H).
template <typename T>
cudaError_t heff_chain_t(mm_problem *p, const void *m, void *H, const double *hext, int mode, cudaStream_t s,
                         double hscale)
{
    const Geom &g = p->g;
    FieldPtrs<T> P = make_ptrs<T>(p);
    P.m_src = (const T *)m;
    P.H_out = (T *)H;
    P.hscale = hscale;
    cudaError_t e = launch_xfwd<T, false>(g, P, s);
    if (e) return e;
    if ((e = launch_conv<T>(g, P, s))) return e;
    if (mode == MODE_HEFF) return launch_xinv<T, MODE_HEFF>(g, P, s, hext, 0, 0);
    return launch_xinv<T, MODE_ENERGY>(g, P, s, hext, 0, 0);
}

template <typename T>
cudaError_t min_body_t(mm_problem *p, cudaGraphConditionalHandle h, cudaStream_t s, int use_cond)
{
    const Geom &g = p->g;
    FieldPtrs<T> P = make_ptrs<T>(p);
    cudaError_t e = launch_xfwd<T, true>(g, P, s);
    if (e) return e;
    if ((e = launch_conv<T>(g, P, s))) return e;
    return launch_xinv<T, MODE_MIN>(g, P, s, nullptr, h, use_cond);
}

template <typename T>
cudaError_t stage_times_t(mm_problem *p, int reps, double *ms, cudaStream_t s)
{
    const Geom &g = p->g;
    FieldPtrs<T> P = make_ptrs<T>(p);
    const int nst = g.bulk ? 5 : 3;
    cudaEvent_t ev[6];
    for (int i = 0; i <= nst; ++i)
        if (cudaEventCreate(&ev[i])) return cudaGetLastError();
    double acc[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && !e; ++r) {
        int i = 0;
        cudaEventRecord(ev[i++], s);
        launch_xfwd<T, true>(g, P, s);
        cudaEventRecord(ev[i++], s);
        if (g.bulk) {
            for (int pass = 0; pass < 3; ++pass) {
                mm_bulk_conv(g, P, s, pass);
                cudaEventRecord(ev[i++], s);
            }
        } else {
            launch_yz_any<T>(g, P, s);
            cudaEventRecord(ev[i++], s);
        }
        launch_xinv<T, MODE_MIN>(g, P, s, nullptr, 0, 0);
        cudaEventRecord(ev[i++], s);
        if ((e = cudaGetLastError())) break;
        if ((e = cudaEventSynchronize(ev[nst]))) break;
        for (int k = 0; k < nst; ++k) {
            float t = 0;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
    }
    for (int i = 0; i <= nst; ++i) cudaEventDestroy(ev[i]);
    for (int i = 0; i < nst; ++i) ms[i] = acc[i] / (reps > 0 ? reps : 1);
    return e;
}

} // namespace

// ---------------------------------------------------------------------------
// exported to api.cu
// ---------------------------------------------------------------------------
#define DISPATCH(p, expr_d, expr_f) ((p)->precision == MM_FP64 ? (expr_d) : (expr_f))


// Shared-memory needs of a launch shape (bytes), for the planner.
size_t mm_smem_x_for(const mm_problem *p, int ty)
{
    Geom g = p->g;
    g.TY = ty;
    return DISPATCH(p, smem_x_t<double>(g), smem_x_t<float>(g));
}
size_t mm_smem_yz_for(const mm_problem *p)
{
    return DISPATCH(p, smem_yz_t<double>(p->g), smem_yz_t<float>(p->g));
}
int mm_yz_thread_bound(const mm_problem *p) { return DISPATCH(p, YZBound<double>::v, YZBound<float>::v); }

int mm_heff_configure(mm_problem *p)
{
    // limits for the largest admissible tile (shared memory grows with it)
    Geom g = p->g;
    g.TY = g.TYF = p->tys[p->nty - 1];
    const size_t sx = DISPATCH(p, smem_x_t<double>(g), smem_x_t<float>(g));
    const size_t sxf = DISPATCH(p, smem_xf_t<double>(g), smem_xf_t<float>(g));
    const size_t syz = p->g.bulk ? 0 : mm_smem_yz_for(p);
    cudaError_t e = DISPATCH(p, configure_t<double>(g, sxf, sx, syz), configure_t<float>(g, sxf, sx, syz));
    if (!e && p->g.bulk) e = mm_bulk_configure(p);
    if (e) { mm_set_cuda_error(e, "cudaFuncSetAttribute"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_autotune(mm_problem *p, const int *tys, int nty, const int *rbs, int nrb, cudaStream_t s)
{
    cudaError_t e = DISPATCH(p, autotune_t<double>(p, tys, nty, rbs, nrb, s),
                             autotune_t<float>(p, tys, nty, rbs, nrb, s));
    if (e) { mm_set_cuda_error(e, "autotune"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_field(mm_problem *p, const void *m, void *H, const double *hext, int mode, cudaStream_t s,
                    double hscale)
{
    cudaError_t e = DISPATCH(p, heff_chain_t<double>(p, m, H, hext, mode, s, hscale),
                             heff_chain_t<float>(p, m, H, hext, mode, s, hscale));
    if (e) { mm_set_cuda_error(e, "field kernels"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_min_body(mm_problem *p, cudaGraphConditionalHandle h, cudaStream_t s, int use_cond)
{
    cudaError_t e = DISPATCH(p, min_body_t<double>(p, h, s, use_cond), min_body_t<float>(p, h, s, use_cond));
    if (e) { mm_set_cuda_error(e, "minimiser body"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_kernel_stage_times(mm_problem *p, int reps, double *ms, const char **names, int *count, cudaStream_t s)
{
    static const char *film[3] = {"xfwd_step", "yz_conv", "xinv_local_bb"};
    static const char *bulk[5] = {"xfwd_step", "y_fwd", "z_conv", "y_inv", "xinv_local_bb"};
    const int nst = p->g.bulk ? 5 : 3;
    if (*count < nst) return MM_ERR_ARG;
    cudaError_t e = DISPATCH(p, stage_times_t<double>(p, reps, ms, s), stage_times_t<float>(p, reps, ms, s));
    if (e) { mm_set_cuda_error(e, "stage timing"); return MM_ERR_CUDA; }
    for (int i = 0; i < nst; ++i) names[i] = p->g.bulk ? bulk[i] : film[i];
    *count = nst;
    return MM_OK;
}

int mm_launch_init_state(mm_problem *p, const double Hext[3], const mm_min_opts *o, int reset_base, cudaStream_t s)
{
    double tau0 = o->tau0 > 0 ? o->tau0 : 1e-2 / p->g.Ms;
    unsigned long long to = o->timeout_s > 0 ? (unsigned long long)(o->timeout_s * 1e9) : 0ull;
    const double kappa = o->tau_kappa > 0 ? o->tau_kappa : 0.5;
    k_init_state<<<1, 32, 0, s>>>(p->st, tau0, o->tol * p->g.Ms, Hext[0], Hext[1], Hext[2], o->max_iter,
                                  o->step_kind, to, reset_base, o->tau_rule, kappa);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_init_state"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_record(mm_problem *p, int step, cudaStream_t s)
{
    k_record<<<1, 32, 0, s>>>(p->st, p->rec_dev, step);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_record"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_copy_result(mm_problem *p, void *dst, cudaStream_t s)
{
    const long n3 = 3 * p->g.N;
    const int blocks = mm_grid_for(n3, 256, 8);
    if (p->precision == MM_FP64)
        k_copy_result<double><<<blocks, 256, 0, s>>>(p->st, (const double *)p->mbuf[0],
                                                    (const double *)p->mbuf[1], (double *)dst, n3);
    else
        k_copy_result<float><<<blocks, 256, 0, s>>>(p->st, (const float *)p->mbuf[0],
                                                   (const float *)p->mbuf[1], (float *)dst, n3);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_copy_result"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_twiddles(mm_problem *p, cudaStream_t s)
{
    const Geom &g = p->g;
    const int L[3] = {g.Px, g.Py, g.Pz};
    void *dst[3] = {p->tw_px, p->tw_py, p->tw_pz};
    for (int i = 0; i < 3; ++i) {
        const int blocks = (L[i] + 255) / 256;
        if (p->precision == MM_FP64) k_twiddle<double><<<blocks, 256, 0, s>>>((double2 *)dst[i], L[i]);
        else k_twiddle<float><<<blocks, 256, 0, s>>>((float2 *)dst[i], L[i]);
    }
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_twiddle"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_convert(mm_problem *p, void *dst, const double *src, long n, cudaStream_t s)
{
    const int blocks = mm_grid_for(n, 256, 8);
    if (p->precision == MM_FP64) k_convert<double><<<blocks, 256, 0, s>>>((double *)dst, src, n);
    else k_convert<float><<<blocks, 256, 0, s>>>((float *)dst, src, n);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_convert"); return MM_ERR_CUDA; }
    return MM_OK;
}
