// Bulk layout of the demagnetisation convolution (Section 3's zero-padded
// FFT convolution for three-dimensional samples).
//
// The film kernel k_yz holds a whole padded y-z plane of one x-frequency in
// shared memory, which bounds nz * Py.  Bulk samples (a cube of 256^3 cells
// pads to 512 x 512 x 512) split that stage into three passes through HBM:
//
//  k_ypass<fwd>  per (kx, ZB z-planes): FFT along y of the three components,
//                zero padding ny -> Py, W[kx][z][y][c] -> W2[kx][z][ky][c];
//  k_zconv       per (kx, KB y-frequencies): FFT along z (padding nz -> Pz),
//                the product with the symmetric 3x3 tensor spectrum
//                (H^ = -Ms N^ m^, normalisation folded into N^), inverse FFT
//                along z keeping the first nz values, in place in W2;
//  k_ypass<inv>  inverse FFT along y keeping the first ny rows, W2 -> W.
//
// The x passes (k_xfwd with the minimiser step, k_xinv with the local terms
// and the step-size sums) are the film kernels unchanged.  Shared-memory rows
// use the padded Stockham layout of fft.cuh.
#include "common.cuh"
#include "fft.cuh"

namespace {

template <typename T> struct BulkBound { static constexpr int v = sizeof(T) == 8 ? 384 : 512; };

template <typename T, bool INV, int LY>
__global__ void __launch_bounds__(BulkBound<T>::v) k_ypass(Geom g, FieldPtrs<T> P)
{
    typedef typename cvec<T>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int ny = g.ny, nz = g.nz, Py = g.Py, ZB = g.ZB, rs = g.rsy;
    const int kx = blockIdx.x, z0 = blockIdx.y * ZB;
    const int zb = min(ZB, nz - z0);
    V *tw = S + 3 * ZB * rs;
    load_twiddles_async(tw, P.tw_py, Py);
    const long first = (long)kx * nz + z0;  // first (kx, z) row pair of this CTA
    const int lin = INV ? Py : ny;           // input length per (z, c) row
    const V *src = INV ? P.W2 + first * Py * 3 : P.W + first * ny * 3;
    // [zl][y][c] -> row (c, zl); PF loads per thread in flight before use
    constexpr int PF = sizeof(T) == 4 ? 8 : 4;
    const int tot = zb * lin * 3;
    for (int e0 = tid; e0 < tot; e0 += PF * nth) {
        V v[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e < tot) v[i] = __ldcg(src + e);
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e >= tot) break;
            const int c = e % 3, rest = e / 3, zl = rest / lin, y = rest - zl * lin;
            S[(c * ZB + zl) * rs + spos<V>(y)] = v[i];
        }
    }
    if (!INV) {
        const int npad = Py - ny;
        for (int e = tid; e < 3 * zb * npad; e += nth) {
            const int r = e / npad, y = ny + (e - r * npad);
            const int c = r / zb, zl = r - c * zb;
            S[(c * ZB + zl) * rs + spos<V>(y)] = czero<V>();
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int Gy = g.Gy, RB = g.RBY;
    const int rb = tid / Gy, j = tid - rb * Gy;
    for (int r0 = 0; r0 < 3 * ZB; r0 += RB) {
        const int r = r0 + rb;
        const bool act = rb < RB && r < 3 * ZB && (r % ZB) < zb;
        fft_row<INV, !INV, INV, 1, LY>(S + (act ? r : 0) * rs, Py, g.lpy, j, tw, act);
    }
    __syncthreads();
    const int lout = INV ? ny : Py;
    V *dst = INV ? P.W + first * ny * 3 : P.W2 + first * Py * 3;
    for (int e = tid; e < zb * lout * 3; e += nth) {
        const int c = e % 3, rest = e / 3, zl = rest / lout, y = rest - zl * lout;
        dst[e] = S[(c * ZB + zl) * rs + spos<V>(y)];
    }
}

template <typename T, int LZ>
__global__ void __launch_bounds__(BulkBound<T>::v) k_zconv(Geom g, FieldPtrs<T> P)
{
    typedef typename cvec<T>::type V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *S = reinterpret_cast<V *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nz = g.nz, Py = g.Py, Pz = g.Pz, KB = g.KB, rs = g.rsz;
    const int kx = blockIdx.x, ky0 = blockIdx.y * KB;
    const int kb = min(KB, Py - ky0);
    V *tw = S + 3 * KB * rs;
    load_twiddles_async(tw, P.tw_pz, Pz);
    // W2[kx][z][ky0 + kyl][c], z < nz -> row (c, kyl), element z; PF loads
    // per thread in flight before use
    V *base = P.W2 + ((long)kx * nz * Py + ky0) * 3;
    const long zs = (long)Py * 3;
    constexpr int PF = sizeof(T) == 4 ? 8 : 4;
    const int tot = nz * kb * 3;
    for (int e0 = tid; e0 < tot; e0 += PF * nth) {
        V v[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e < tot) {
                const int c = e % 3, rest = e / 3, kyl = rest % kb, z = rest / kb;
                v[i] = __ldcg(base + (long)z * zs + kyl * 3 + c);
            }
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int e = e0 + i * nth;
            if (e >= tot) break;
            const int c = e % 3, rest = e / 3, kyl = rest % kb, z = rest / kb;
            S[(c * KB + kyl) * rs + spos<V>(z)] = v[i];
        }
    }
    const int npad = Pz - nz;
    for (int e = tid; e < 3 * kb * npad; e += nth) {
        const int r = e / npad, z = nz + (e - r * npad);
        const int c = r / kb, kyl = r - c * kb;
        S[(c * KB + kyl) * rs + spos<V>(z)] = czero<V>();
    }
    cp_async_wait_all();
    __syncthreads();
    const int Gz = g.Gz, RB = g.RBZ;
    const int rb = tid / Gz, j = tid - rb * Gz;
    for (int r0 = 0; r0 < 3 * KB; r0 += RB) {
        const int r = r0 + rb;
        const bool act = rb < RB && r < 3 * KB && (r % KB) < kb;
        fft_row<false, true, false, 1, LZ>(S + (act ? r : 0) * rs, Pz, g.lpz, j, tw, act);
    }
    __syncthreads();
    // tensor product per (ky, kz); octant storage [kx][kzr][kyr][6] with the
    // off-diagonal signs of the reflected frequencies
    const int hy = Py / 2, hz = Pz / 2;
    const T *Nk = P.Nhat + (long)kx * (hz + 1) * (hy + 1) * 6;
    for (int e = tid; e < kb * Pz; e += nth) {
        const int kyl = e % kb, kz = e / kb, ky = ky0 + kyl;
        const int kyr = ky <= hy ? ky : Py - ky, kzr = kz <= hz ? kz : Pz - kz;
        const T sy = ky <= hy ? (T)1 : (T)-1, sz = kz <= hz ? (T)1 : (T)-1;
        const T *n6 = Nk + ((long)kzr * (hy + 1) + kyr) * 6;
        const T nxx = __ldg(n6 + 0), nyy = __ldg(n6 + 1), nzz = __ldg(n6 + 2);
        const T nxy = sy * __ldg(n6 + 3), nxz = sz * __ldg(n6 + 4), nyz = sy * sz * __ldg(n6 + 5);
        V *a0 = S + (0 * KB + kyl) * rs + spos<V>(kz);
        V *a1 = S + (1 * KB + kyl) * rs + spos<V>(kz);
        V *a2 = S + (2 * KB + kyl) * rs + spos<V>(kz);
        const V m0 = *a0, m1 = *a1, m2 = *a2;
        V h0, h1, h2;
        h0.x = nxx * m0.x + nxy * m1.x + nxz * m2.x; h0.y = nxx * m0.y + nxy * m1.y + nxz * m2.y;
        h1.x = nxy * m0.x + nyy * m1.x + nyz * m2.x; h1.y = nxy * m0.y + nyy * m1.y + nyz * m2.y;
        h2.x = nxz * m0.x + nyz * m1.x + nzz * m2.x; h2.y = nxz * m0.y + nyz * m1.y + nzz * m2.y;
        *a0 = h0; *a1 = h1; *a2 = h2;
    }
    __syncthreads();
    for (int r0 = 0; r0 < 3 * KB; r0 += RB) {
        const int r = r0 + rb;
        const bool act = rb < RB && r < 3 * KB && (r % KB) < kb;
        fft_row<true, false, true, 1, LZ>(S + (act ? r : 0) * rs, Pz, g.lpz, j, tw, act);
    }
    __syncthreads();
    for (int e = tid; e < nz * kb * 3; e += nth) {
        const int c = e % 3, rest = e / 3, kyl = rest % kb, z = rest / kb;
        base[(long)z * zs + kyl * 3 + c] = S[(c * KB + kyl) * rs + spos<V>(z)];
    }
}

inline int round32(int n) { return (n + 31) & ~31; }

template <typename T> size_t smem_y_t(const Geom &g, int zb)
{
    typedef typename cvec<T>::type V;
    return ((size_t)3 * zb * g.rsy + g.Py) * sizeof(V);
}
template <typename T> size_t smem_z_t(const Geom &g, int kb)
{
    typedef typename cvec<T>::type V;
    return ((size_t)3 * kb * g.rsz + g.Pz) * sizeof(V);
}

inline int lc_of(int logL) { return MM_FFT_SPECIALISED(logL) ? logL : 0; }
#define MM_LC_CASES(X) X(0) X(6) X(7) X(8) X(9) X(10)

template <typename T> cudaError_t bulk_conv_t(const Geom &g, const FieldPtrs<T> &P, cudaStream_t s, int pass)
{
    const dim3 gy(g.C, (g.nz + g.ZB - 1) / g.ZB), gz(g.C, (g.Py + g.KB - 1) / g.KB);
    const int ty = round32(g.RBY * g.Gy), tz = round32(g.RBZ * g.Gz);
    const size_t sy = smem_y_t<T>(g, g.ZB), sz = smem_z_t<T>(g, g.KB);
    const int ly = lc_of(g.lpy), lz = lc_of(g.lpz);
    if (pass < 0 || pass == 0) {
        switch (ly) {
#define C(L) case L: k_ypass<T, false, L><<<gy, ty, sy, s>>>(g, P); break;
            MM_LC_CASES(C)
#undef C
        }
    }
    if (pass < 0 || pass == 1) {
        switch (lz) {
#define C(L) case L: k_zconv<T, L><<<gz, tz, sz, s>>>(g, P); break;
            MM_LC_CASES(C)
#undef C
        }
    }
    if (pass < 0 || pass == 2) {
        switch (ly) {
#define C(L) case L: k_ypass<T, true, L><<<gy, ty, sy, s>>>(g, P); break;
            MM_LC_CASES(C)
#undef C
        }
    }
    return cudaGetLastError();
}

// the bytes a launch needs must fit the common cap, which every kernel is given
template <typename F> cudaError_t smem_attr(F *f, size_t bytes)
{
    if (bytes > (size_t)MM_SMEM_CAP) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM_CAP);
}

template <typename T> cudaError_t configure_t(const Geom &g)
{
    cudaError_t e = cudaSuccess;
    const size_t sy = smem_y_t<T>(g, g.ZB), sz = smem_z_t<T>(g, g.KB);
    switch (lc_of(g.lpy)) {
#define C(L) case L: if ((e = smem_attr(k_ypass<T, false, L>, sy)) || (e = smem_attr(k_ypass<T, true, L>, sy))) return e; break;
        MM_LC_CASES(C)
#undef C
    }
    switch (lc_of(g.lpz)) {
#define C(L) case L: return smem_attr(k_zconv<T, L>, sz);
        MM_LC_CASES(C)
#undef C
    }
    return cudaErrorInvalidValue;
}

} // namespace

cudaError_t mm_bulk_conv(const Geom &g, const FieldPtrs<double> &P, cudaStream_t s, int pass)
{
    return bulk_conv_t<double>(g, P, s, pass);
}
cudaError_t mm_bulk_conv(const Geom &g, const FieldPtrs<float> &P, cudaStream_t s, int pass)
{
    return bulk_conv_t<float>(g, P, s, pass);
}

size_t mm_bulk_smem_y(const mm_problem *p, int zb)
{
    return p->precision == MM_FP64 ? smem_y_t<double>(p->g, zb) : smem_y_t<float>(p->g, zb);
}
size_t mm_bulk_smem_z(const mm_problem *p, int kb)
{
    return p->precision == MM_FP64 ? smem_z_t<double>(p->g, kb) : smem_z_t<float>(p->g, kb);
}
int mm_bulk_thread_bound(const mm_problem *p)
{
    return p->precision == MM_FP64 ? BulkBound<double>::v : BulkBound<float>::v;
}
cudaError_t mm_bulk_configure(const mm_problem *p)
{
    return p->precision == MM_FP64 ? configure_t<double>(p->g) : configure_t<float>(p->g);
}
