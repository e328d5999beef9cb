// Demagnetisation tensor setup (once per geometry).
//
// The demagnetisation field of Section 3 is a discrete convolution with the
// cell-averaged tensor of Newell, Williams and Dunlop (J. Geophys. Res. 98
// (1993) 9551):
//   N_xx(X,Y,Z) = 1/(4 pi dx dy dz) sum_{e in {-1,0,1}^3} c(e) f(X+e1 dx, Y+e2 dy, Z+e3 dz),
//   c(e) = 8, -4, 2, -1 for 0, 1, 2, 3 non-zero entries of e,
// N_yy, N_zz by permuting coordinates, N_xy, N_xz, N_yz likewise from g.
//
//  k_newell_table    f and g (six permutations) on the (nx+1)(ny+1)(nz+1)
//                    non-negative lattice, in double-double (dd.cuh): the
//                    second difference cancels ~R^6 of their magnitude.
//  k_newell_stencil  the 27-point sums in double-double, rounded to double:
//                    the first octant of offsets, [6][nz][ny][nx].
//  k_place / k_fft_strided / k_extract
//                    the tensor placed circularly on the zero-padded grid
//                    (offsets -(n-1)..(n-1), unused entries 0), its 3-D FFT in
//                    double, and the real parts (all six spectra are real by
//                    the even/odd symmetry) of the octant kx <= Px/2,
//                    ky <= Py/2, kz <= Pz/2, scaled by -Ms/(Px Py Pz) so that
//                    the convolution kernels need no other normalisation.
#include "common.cuh"
#include "dd.cuh"
#include "fft.cuh"

namespace {

__global__ void k_newell_table(int nx, int ny, int nz, double hx, double hy, double hz, dd_t *T)
{
    const long ax = nx + 1, ay = ny + 1, az = nz + 1, na = ax * ay * az;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < na; p += (long)gridDim.x * blockDim.x) {
        const long a = p % ax, b = (p / ax) % ay, c = p / (ax * ay);
        // lattice coordinates are exact in dd: integer times a double
        const dd_t X = dd_two_prod((double)a, hx), Y = dd_two_prod((double)b, hy), Z = dd_two_prod((double)c, hz);
        T[0 * na + p] = dd_newell_f(X, Y, Z);
        T[1 * na + p] = dd_newell_f(Y, X, Z);
        T[2 * na + p] = dd_newell_f(Z, Y, X);
        T[3 * na + p] = dd_newell_g(X, Y, Z);
        T[4 * na + p] = dd_newell_g(X, Z, Y);
        T[5 * na + p] = dd_newell_g(Y, Z, X);
    }
}

__global__ void k_newell_stencil(int nx, int ny, int nz, double hx, double hy, double hz, const dd_t *T,
                                 double *out)
{
    const long ax = nx + 1, ay = ny + 1, az = nz + 1, na = ax * ay * az;
    const long nn = (long)nx * ny * nz;
    // 1 / (4 pi hx hy hz) in dd
    const dd_t pi = dd_make(DD_PI_HI, DD_PI_LO);
    const dd_t vol = dd_mul(dd_mul(dd_from(hx), dd_from(hy)), dd_from(hz));
    const dd_t norm = dd_div(dd_from(1.0), dd_mul(dd_ldexp(pi, 2), vol));
    const int W[4] = {8, -4, 2, -1};
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < nn; p += (long)gridDim.x * blockDim.x) {
        const long i = p % nx, j = (p / nx) % ny, k = p / ((long)nx * ny);
        dd_t s[6];
        for (int c = 0; c < 6; ++c) s[c] = dd_from(0.0);
        for (int e1 = -1; e1 <= 1; ++e1)
            for (int e2 = -1; e2 <= 1; ++e2)
                for (int e3 = -1; e3 <= 1; ++e3) {
                    const double w = (double)W[(e1 != 0) + (e2 != 0) + (e3 != 0)];
                    const long a = i + e1, b = j + e2, c3 = k + e3;
                    const long q = ((c3 < 0 ? -c3 : c3) * ay + (b < 0 ? -b : b)) * ax + (a < 0 ? -a : a);
                    const double sa = a < 0 ? -1.0 : 1.0, sb = b < 0 ? -1.0 : 1.0, sc = c3 < 0 ? -1.0 : 1.0;
                    s[0] = dd_add(s[0], dd_mul_d(T[0 * na + q], w));
                    s[1] = dd_add(s[1], dd_mul_d(T[1 * na + q], w));
                    s[2] = dd_add(s[2], dd_mul_d(T[2 * na + q], w));
                    s[3] = dd_add(s[3], dd_mul_d(T[3 * na + q], w * sa * sb));  // g(x,y,z): odd in x, y
                    s[4] = dd_add(s[4], dd_mul_d(T[4 * na + q], w * sa * sc));  // g(x,z,y): odd in x, z
                    s[5] = dd_add(s[5], dd_mul_d(T[5 * na + q], w * sb * sc));  // g(y,z,x): odd in y, z
                }
        for (int c = 0; c < 6; ++c) {
            const dd_t v = dd_mul(s[c], norm);
            out[c * nn + p] = v.hi + v.lo;
        }
    }
}

// parity of component c under sign flips of the x, y, z offsets
__device__ __forceinline__ double comp_sign(int c, long i, long j, long k)
{
    const bool nx_ = i < 0, ny_ = j < 0, nz_ = k < 0;
    bool flip = false;
    if (c == 3) flip = nx_ ^ ny_;
    else if (c == 4) flip = nx_ ^ nz_;
    else if (c == 5) flip = ny_ ^ nz_;
    return flip ? -1.0 : 1.0;
}

__global__ void k_place(int c, int nx, int ny, int nz, int Px, int Py, int Pz, const double *Noct, double2 *F)
{
    const long tot = (long)Px * Py * Pz;
    const long nn = (long)nx * ny * nz;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < tot; p += (long)gridDim.x * blockDim.x) {
        const long ii = p % Px, jj = (p / Px) % Py, kk = p / ((long)Px * Py);
        const long i = ii < nx ? ii : (ii > Px - nx ? ii - Px : Px);
        const long j = jj < ny ? jj : (jj > Py - ny ? jj - Py : Py);
        const long k = kk < nz ? kk : (kk > Pz - nz ? kk - Pz : Pz);
        double v = 0.0;
        if (i != Px && j != Py && k != Pz) {
            const long ai = i < 0 ? -i : i, aj = j < 0 ? -j : j, ak = k < 0 ? -k : k;
            v = comp_sign(c, i, j, k) * Noct[c * nn + (ak * ny + aj) * nx + ai];
        }
        F[p] = make_double2(v, 0.0);
    }
}

__global__ void k_twiddle_d(double2 *tw, int L)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)L, &s, &c);
    tw[t] = make_double2(c, -s);
}

// Forward FFT of rows of length L along a strided axis: row r starts at
// base(r) = (r % inner) + (r / inner) * outer_stride and its elements are
// `stride` apart.  One CTA per row.
__global__ void k_fft_strided(double2 *F, int L, int logL, long stride, long inner, long outer_stride,
                              const double2 *tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *S = reinterpret_cast<double2 *>(smem_raw);
    const long r = blockIdx.x;
    const long base = (r % inner) + (r / inner) * outer_stride;
    for (int t = threadIdx.x; t < L; t += blockDim.x) S[pidx(t)] = F[base + t * stride];
    __syncthreads();
    const int G = L >= 8 ? L / 8 : 1;
    const bool act = threadIdx.x < G;
    fft_row<false, false, false, 1, 0>(S, L, logL, act ? (int)threadIdx.x : 0, tw, act);
    __syncthreads();
    for (int t = threadIdx.x; t < L; t += blockDim.x) F[base + t * stride] = S[pidx(t)];
}

template <typename T>
__global__ void k_extract(int c, int Px, int Py, int Pz, const double2 *F, double scale, T *Nhat)
{
    const int hx = Px / 2, hy = Py / 2, hz = Pz / 2;
    const long tot = (long)(hx + 1) * (hy + 1) * (hz + 1);
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < tot; p += (long)gridDim.x * blockDim.x) {
        const long ky = p % (hy + 1), kz = (p / (hy + 1)) % (hz + 1), kx = p / ((long)(hy + 1) * (hz + 1));
        const double v = F[(kz * Py + ky) * Px + kx].x;
        Nhat[p * 6 + c] = (T)(scale * v);
    }
}

// Film layout: the tensor transformed along x and y only, at real z offsets
// dz = 0 .. nzf-1 with nzf = max(1, Pz/2) (zero for dz >= nz), for the
// direct z-convolution of the film kernel: K[kx][dz][c][ky], kx <= Px/2,
// ky <= Py/2, scaled by -Ms/(Px Py).  The xx, yy, zz and xy transforms are
// real, the xz and yz transforms imaginary (odd in x or y and in z); their
// imaginary parts are stored, and zero at dz = 0.
template <typename T>
__global__ void k_extract_film(int c, int Px, int Py, int nz, int nzf, const double2 *F, double scale, T *K)
{
    const int hx = Px / 2, hy = Py / 2;
    const long tot = (long)(hx + 1) * nzf * (hy + 1);
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < tot; p += (long)gridDim.x * blockDim.x) {
        const long ky = p % (hy + 1), dz = (p / (hy + 1)) % nzf, kx = p / ((long)(hy + 1) * nzf);
        double v = 0.0;
        if (dz < nz) {
            const double2 f = F[(dz * Py + ky) * Px + kx];
            v = c < 4 ? f.x : (dz == 0 ? 0.0 : f.y);
        }
        K[((kx * nzf + dz) * 6 + c) * (hy + 1) + ky] = (T)(scale * v);
    }
}

int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

} // namespace

// Newell octant on the device: N_dev [6][nz][ny][nx] doubles.
int mm_newell_device(const mm_grid *gr, double *N_dev, cudaStream_t s)
{
    double h = gr->dx;
    if (gr->dy > h) h = gr->dy;
    if (gr->dz > h) h = gr->dz;
    const double hx = gr->dx / h, hy = gr->dy / h, hz = gr->dz / h;
    const long na = (long)(gr->nx + 1) * (gr->ny + 1) * (gr->nz + 1);
    const long nn = (long)gr->nx * gr->ny * gr->nz;
    dd_t *T = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&T, sizeof(dd_t) * 6 * (size_t)na, s);
    if (e) { mm_set_cuda_error(e, "cudaMallocAsync(newell table)"); return MM_ERR_OOM; }
    const int bt = 128;
    long blocks = (na + bt - 1) / bt;
    if (blocks > mm_sm_count() * 64L) blocks = mm_sm_count() * 64L;
    k_newell_table<<<(int)blocks, bt, 0, s>>>(gr->nx, gr->ny, gr->nz, hx, hy, hz, T);
    e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "mm_newell_static table kernel"); return MM_ERR_CUDA; }
    blocks = (nn + bt - 1) / bt;
    if (blocks > mm_sm_count() * 64L) blocks = mm_sm_count() * 64L;
    k_newell_stencil<<<(int)blocks, bt, 0, s>>>(gr->nx, gr->ny, gr->nz, hx, hy, hz, T, N_dev);
    e = cudaGetLastError();
    cudaFreeAsync(T, s);
    if (e) { mm_set_cuda_error(e, "newell kernels"); return MM_ERR_CUDA; }
    return MM_OK;
}

// Tensor spectra into p->Nhat in the precision of p: bulk layout
// [Px/2+1][Pz/2+1][Py/2+1][6] (3-D transform, octant); film layout
// [Px/2+1][max(1, Pz/2)][6][Py/2+1] (x-y transform at real z offsets,
// k_extract_film).
int mm_tensor_spectrum(mm_problem *p, const double *N_dev, cudaStream_t s)
{
    const Geom &g = p->g;
    const long tot = (long)g.Px * g.Py * g.Pz;
    double2 *F = nullptr, *tw = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&F, sizeof(double2) * tot, s);
    if (e) { mm_set_cuda_error(e, "cudaMallocAsync(tensor fft)"); return MM_ERR_OOM; }
    e = cudaMallocAsync((void **)&tw, sizeof(double2) * (g.Px + g.Py + g.Pz), s);
    if (e) { cudaFreeAsync(F, s); mm_set_cuda_error(e, "cudaMallocAsync(twiddles)"); return MM_ERR_OOM; }
    double2 *twx = tw, *twy = tw + g.Px, *twz = tw + g.Px + g.Py;
    k_twiddle_d<<<(g.Px + 255) / 256, 256, 0, s>>>(twx, g.Px);
    k_twiddle_d<<<(g.Py + 255) / 256, 256, 0, s>>>(twy, g.Py);
    k_twiddle_d<<<(g.Pz + 255) / 256, 256, 0, s>>>(twz, g.Pz);
    const double scale = -g.Ms / ((double)g.Px * g.Py * g.Pz);
    const int L[3] = {g.Px, g.Py, g.Pz};
    const long stride[3] = {1, g.Px, (long)g.Px * g.Py};
    const long rows[3] = {(long)g.Py * g.Pz, (long)g.Px * g.Pz, (long)g.Px * g.Py};
    // row r -> base: x: r*Px; y: (r % Px) + (r / Px) * Px*Py; z: r
    const long inner[3] = {1, g.Px, (long)g.Px * g.Py};
    const long outer[3] = {g.Px, (long)g.Px * g.Py, 0};
    const double2 *tws[3] = {twx, twy, twz};
    long blocks = (tot + 255) / 256;
    if (blocks > mm_sm_count() * 32L) blocks = mm_sm_count() * 32L;
    const long ext = (long)(g.Px / 2 + 1) * (g.Py / 2 + 1) * (g.Pz / 2 + 1);
    long eblocks = (ext + 255) / 256;
    if (eblocks > mm_sm_count() * 32L) eblocks = mm_sm_count() * 32L;
    // film layout: transforms along x and y only (the film kernel convolves z directly)
    const int naxes = g.bulk ? 3 : 2;
    const int nzf = g.Pz > 1 ? g.Pz / 2 : 1;
    const long fext = (long)(g.Px / 2 + 1) * nzf * (g.Py / 2 + 1);
    long fblocks = (fext + 255) / 256;
    if (fblocks > mm_sm_count() * 32L) fblocks = mm_sm_count() * 32L;
    for (int c = 0; c < 6 && !e; ++c) {
        k_place<<<(int)blocks, 256, 0, s>>>(c, g.nx, g.ny, g.nz, g.Px, g.Py, g.Pz, N_dev, F);
        for (int a = 0; a < naxes; ++a) {
            if (L[a] == 1) continue;
            const int thr = ((L[a] >= 8 ? L[a] / 8 : 1) + 31) & ~31;
            const size_t sm = sizeof(double2) * padded_row(L[a]);
            if (sm > 48 * 1024)
                cudaFuncSetAttribute(k_fft_strided, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_fft_strided<<<(unsigned)rows[a], thr, sm, s>>>(F, L[a], ilog2(L[a]), stride[a], inner[a],
                                                             outer[a] ? outer[a] : 1, tws[a]);
        }
        if (!g.bulk) {
            const double fscale = -g.Ms / ((double)g.Px * g.Py);
            if (p->precision == MM_FP64)
                k_extract_film<double><<<(int)fblocks, 256, 0, s>>>(c, g.Px, g.Py, g.nz, nzf, F, fscale, (double *)p->Nhat);
            else if (p->precision == MM_F32X2)
                k_extract_film<dfloat><<<(int)fblocks, 256, 0, s>>>(c, g.Px, g.Py, g.nz, nzf, F, fscale, (dfloat *)p->Nhat);
            else
                k_extract_film<float><<<(int)fblocks, 256, 0, s>>>(c, g.Px, g.Py, g.nz, nzf, F, fscale, (float *)p->Nhat);
        } else if (p->precision == MM_FP64) {
            k_extract<double><<<(int)eblocks, 256, 0, s>>>(c, g.Px, g.Py, g.Pz, F, scale, (double *)p->Nhat);
        } else {
            k_extract<float><<<(int)eblocks, 256, 0, s>>>(c, g.Px, g.Py, g.Pz, F, scale, (float *)p->Nhat);
        }
        e = cudaGetLastError();
    }
    cudaFreeAsync(F, s);
    cudaFreeAsync(tw, s);
    if (e) { mm_set_cuda_error(e, "tensor spectrum"); return MM_ERR_CUDA; }
    return MM_OK;
}

// ---------------------------------------------------------------------------
// mm_newell_static: the Newell tensor without any device allocation.
//
// Some callers cannot allocate device memory: a process whose memory is
// fully reserved up front by another allocator (a framework's caching pool
// or a fixed per-process budget), or code on a latency-critical stream where
// cudaMalloc/cudaFree, which can synchronise the whole device, are not
// allowed.  For them the double-double table of f and g lives in this
// file-scope device array instead of a cudaMallocAsync buffer.  The array is
// part of the library's image, so every GPU that loads libmmgb.so holds it
// (6 MiB) until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

#define MM_NEWELL_STATIC_POINTS 65536L  // (nx+1)(ny+1)(nz+1) lattice points, six dd values each

static __device__ __align__(256) dd_t g_newell_static_table[6 * MM_NEWELL_STATIC_POINTS];

namespace {
std::mutex g_static_mutex;
void *g_static_addr[256];  // device address of the table, per device ordinal
}

extern "C" MM_API int mm_newell_static(const mm_grid *gr, double *N_dev, void *stream)
{
    if (!gr || !N_dev || gr->nx < 1 || gr->ny < 1 || gr->nz < 1 || !(gr->dx > 0) || !(gr->dy > 0) ||
        !(gr->dz > 0) || !isfinite(gr->dx) || !isfinite(gr->dy) || !isfinite(gr->dz))
        return MM_ERR_ARG;
    // lattice points in 64-bit arithmetic: nx + 1 must not overflow int
    const long na = ((long)gr->nx + 1) * ((long)gr->ny + 1) * ((long)gr->nz + 1);
    if (na > MM_NEWELL_STATIC_POINTS) return MM_ERR_UNSUPPORTED;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, N_dev) != cudaSuccess) { cudaGetLastError(); return MM_ERR_ARG; }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return MM_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) { mm_set_cuda_error(e, "cudaGetDevice"); return MM_ERR_CUDA; }
    if (dev < 0 || dev >= 256) return MM_ERR_UNSUPPORTED;
    // the kernels run on the current device: the output must live there
    if (a.type == cudaMemoryTypeDevice && a.device != dev) return MM_ERR_ARG;
    dd_t *T = nullptr;
    {
        // first call on this device: look up the device address of the table
        // (in host code the array's name is only a host-side stand-in)
        std::lock_guard<std::mutex> lk(g_static_mutex);
        if (!g_static_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_newell_static_table);
            if (e) { mm_set_cuda_error(e, "cudaGetSymbolAddress"); return MM_ERR_CUDA; }
            g_static_addr[dev] = p;
        }
        T = static_cast<dd_t *>(g_static_addr[dev]);
    }
    double h = gr->dx;
    if (gr->dy > h) h = gr->dy;
    if (gr->dz > h) h = gr->dz;
    const double hx = gr->dx / h, hy = gr->dy / h, hz = gr->dz / h;
    const long nn = (long)gr->nx * gr->ny * gr->nz;
    cudaStream_t s = (cudaStream_t)stream;
    const int bt = 128;
    long blocks = (na + bt - 1) / bt;
    if (blocks > mm_sm_count() * 64L) blocks = mm_sm_count() * 64L;
    // every table entry read by the stencil is written first, so nothing needs clearing
    k_newell_table<<<(int)blocks, bt, 0, s>>>(gr->nx, gr->ny, gr->nz, hx, hy, hz, T);
    e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "mm_newell_static table kernel"); return MM_ERR_CUDA; }
    blocks = (nn + bt - 1) / bt;
    if (blocks > mm_sm_count() * 64L) blocks = mm_sm_count() * 64L;
    k_newell_stencil<<<(int)blocks, bt, 0, s>>>(gr->nx, gr->ny, gr->nz, hx, hy, hz, T, N_dev);
    e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "mm_newell_static kernels"); return MM_ERR_CUDA; }
    return MM_OK;
}
