// Tau-orthogonal phase kernels (Sec. 4, App. A): vorticity, separable filter
// passes, enstrophy sensitivities, the QoI / Gram block reduction, the LRS
// history matvec and the single-block FP64 coefficient solve.
//
// Fields are FP32 structure-of-arrays [comp][nz][ny][nx].  Every field is
// zero on solid rows, which is exactly the zero extension the filters and the
// central differences use beyond the walls (Sec. 4.1).
#include "lbm_common.cuh"
#include "rng.cuh"
#include "dfloat.cuh"

namespace lbm {

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ int modp(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// ------------------------------------------------------------ vorticity --
// omega = curl v* by central differences: 3-D (d_y v_z - d_z v_y, d_z v_x -
// d_x v_z, d_x v_y - d_y v_x); 2-D the scalar d_x v_y - d_y v_x.  Written
// after the d velocity components of the stacked field x6.
__global__ void __launch_bounds__(256) curl_kernel(Params p, float* __restrict__ x6) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n, nx = p.nx, ny = p.ny, nz = p.nz;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    const int d = p.dim;
    if (p.walls && (y == 0 || y == ny - 1)) {
        for (int c = d; c < p.ncomp; ++c) x6[(size_t)c * N + n] = 0.f;
        return;
    }
    const int xm = wrapi(x - 1, nx), xp = wrapi(x + 1, nx);
    const int ym = wrapi(y - 1, ny), yp = wrapi(y + 1, ny);
    const size_t r0 = ((size_t)z * ny + y) * nx;
    const size_t iym = ((size_t)z * ny + ym) * nx + x, iyp = ((size_t)z * ny + yp) * nx + x;
    const float* vx = x6;
    const float* vy = x6 + N;
    if (d == 2) {
        const float dxvy = 0.5f * (vy[r0 + xp] - vy[r0 + xm]);
        const float dyvx = 0.5f * (vx[iyp] - vx[iym]);
        x6[(size_t)2 * N + n] = dxvy - dyvx;
        return;
    }
    const float* vz = x6 + 2 * (size_t)N;
    const int zm = wrapi(z - 1, nz), zp = wrapi(z + 1, nz);
    const size_t izm = ((size_t)zm * ny + y) * nx + x, izp = ((size_t)zp * ny + y) * nx + x;
    const float dyvz = 0.5f * (vz[iyp] - vz[iym]), dzvy = 0.5f * (vy[izp] - vy[izm]);
    const float dzvx = 0.5f * (vx[izp] - vx[izm]), dxvz = 0.5f * (vz[r0 + xp] - vz[r0 + xm]);
    const float dxvy = 0.5f * (vy[r0 + xp] - vy[r0 + xm]), dyvx = 0.5f * (vx[iyp] - vx[iym]);
    x6[(size_t)3 * N + n] = dyvz - dzvy;
    x6[(size_t)4 * N + n] = dzvx - dxvz;
    x6[(size_t)5 * N + n] = dxvy - dyvx;
}

// --------------------------------------------------------- filter pass --
// out(x) = [out(x) +] scale * sum_r t(r) in(x - r e_axis) for every component:
// one 1-D factor of a separable filter.  Periodic along x and z (and y without
// walls, any radius); along y with walls, rows outside the array contribute
// nothing and solid rows hold zero, and the output is zero on solid rows.
__global__ void __launch_bounds__(256) pass_kernel(Params p, const float* __restrict__ in, float* __restrict__ out,
                                                   int ncomp, int axis, Taps tp, float scale, int accumulate) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const size_t N = (size_t)p.n;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    if (p.walls && (y == 0 || y == ny - 1)) {
        for (int c = 0; c < ncomp; ++c) out[c * N + n] = 0.f;
        return;
    }
    const int R = tp.radius;
    for (int c = 0; c < ncomp; ++c) {
        const float* a = in + c * N;
        float s = 0.f;
        if (axis == 0) {
            const size_t row = ((size_t)z * ny + y) * nx;
            for (int r = -R; r <= R; ++r) s += tp.t[r + R] * a[row + modp(x - r, nx)];
        } else if (axis == 1) {
            if (p.walls) {
                for (int r = -R; r <= R; ++r) {
                    const int ys = y - r;
                    if (ys >= 0 && ys < ny) s += tp.t[r + R] * a[((size_t)z * ny + ys) * nx + x];
                }
            } else {
                for (int r = -R; r <= R; ++r) s += tp.t[r + R] * a[((size_t)z * ny + modp(y - r, ny)) * nx + x];
            }
        } else {
            for (int r = -R; r <= R; ++r) s += tp.t[r + R] * a[((size_t)modp(z - r, nz) * ny + y) * nx + x];
        }
        float* o = out + c * N + n;
        *o = accumulate ? (*o + scale * s) : scale * s;
    }
}

// ------------------------------------------------------- Fourier bands --
// out = in * (1/(nx ny) if lo - 1/2 <= |k| < hi + 1/2 else 0) on the R2C half
// spectrum [c][ky][kx] (kx = 0..nx/2, ky folded to -ny/2..ny/2-1): the sharp
// filter R_[lo,hi] of Sec. 4.1 with the inverse transform's normalisation.
// The band edges sit at half-integers, so the test on the integer |k|^2 is exact.
__global__ void __launch_bounds__(256) band_mask_kernel(Params p, const float2* __restrict__ in,
                                                        float2* __restrict__ out, int ncomp, int lo, int hi) {
    const int nxh = p.nx / 2 + 1;
    const long long per = (long long)p.ny * nxh;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per * ncomp) return;
    const long long e = i % per;
    const int kx = (int)(e % nxh);
    const int jy = (int)(e / nxh);
    const int ky = jy <= p.ny / 2 ? jy : jy - p.ny;
    const long long k2 = (long long)kx * kx + (long long)ky * ky;
    // lo - 1/2 <= |k|  <=>  k2 >= lo^2 - lo + 1 (lo >= 1);  |k| < hi + 1/2  <=>  k2 <= hi^2 + hi
    const bool keep = (lo == 0 || k2 >= (long long)lo * lo - lo + 1) && k2 <= (long long)hi * hi + hi;
    const float sc = keep ? 1.0f / ((float)p.nx * (float)p.ny) : 0.f;
    const float2 v = in[i];
    out[i] = make_float2(v.x * sc, v.y * sc);
}

// ---------------------------------------------- enstrophy sensitivities --
// V_Z = curl*(W), W = R R omega (App. A): 2-D (d_y W, -d_x W); 3-D curl W.
__global__ void __launch_bounds__(256) sens_curl_kernel(Params p, const float* __restrict__ w, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n, nx = p.nx, ny = p.ny, nz = p.nz;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    const int d = p.dim;
    if (p.walls && (y == 0 || y == ny - 1)) {
        for (int c = 0; c < d; ++c) out[(size_t)c * N + n] = 0.f;
        return;
    }
    const int xm = wrapi(x - 1, nx), xp = wrapi(x + 1, nx);
    const int ym = wrapi(y - 1, ny), yp = wrapi(y + 1, ny);
    const size_t r0 = ((size_t)z * ny + y) * nx;
    const size_t iym = ((size_t)z * ny + ym) * nx + x, iyp = ((size_t)z * ny + yp) * nx + x;
    if (d == 2) {
        out[n] = 0.5f * (w[iyp] - w[iym]);
        out[(size_t)N + n] = -0.5f * (w[r0 + xp] - w[r0 + xm]);
        return;
    }
    const float* wx = w;
    const float* wy = w + N;
    const float* wz = w + 2 * (size_t)N;
    const int zm = wrapi(z - 1, nz), zp = wrapi(z + 1, nz);
    const size_t izm = ((size_t)zm * ny + y) * nx + x, izp = ((size_t)zp * ny + y) * nx + x;
    out[n] = 0.5f * (wz[iyp] - wz[iym]) - 0.5f * (wy[izp] - wy[izm]);
    out[(size_t)N + n] = 0.5f * (wx[izp] - wx[izm]) - 0.5f * (wz[r0 + xp] - wz[r0 + xm]);
    out[(size_t)2 * N + n] = 0.5f * (wy[r0 + xp] - wy[r0 + xm]) - 0.5f * (wx[iyp] - wx[iym]);
}

// ------------------------------------------------------ block reduction --
// Per block (one y row, a chunk of z planes): <v*, V_k> and <V_i, V_j> (i <= j)
// over its fluid nodes, and the row sums of v*_x and V_k,x (the mean-profile
// couplings).  FP32 throughout the block (per thread over a few nodes, then a
// warp tree); the partials are summed with compensation in the solve.  No
// double-precision arithmetic here: on this GPU an FP64 warp tree over the
// NV values of every block costs more than the whole field traversal.
struct RedPtrs {
    const float* v[kMaxQoi];
};

template <int NS>
__global__ void __launch_bounds__(128) reduce_kernel(Params p, const float* __restrict__ vps, RedPtrs vk,
                                                     float* __restrict__ part, float* __restrict__ plane_part) {
    constexpr int NG = NS * (NS + 1) / 2;
    constexpr int NV = NS + NG + 1 + NS;  // <v,V_k>, Gram, row sums (v_x, V_k,x)
    const int y = blockIdx.x;
    const int zc = blockIdx.y;
    const int zper = (p.nz + p.nzc - 1) / p.nzc;
    const int z0 = zc * zper;
    const int z1 = min(p.nz, z0 + zper);
    const size_t N = (size_t)p.n;
    const int d = p.dim;
    float acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.f;
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    const int cnt = solid ? 0 : (z1 - z0) * p.nx;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int z = z0 + e / p.nx;
        const int x = e % p.nx;
        const size_t n = ((size_t)z * p.ny + y) * p.nx + x;
        float u[3], w[NS][3];
        u[0] = vps[n]; u[1] = vps[N + n]; u[2] = d == 3 ? vps[2 * N + n] : 0.f;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            w[k][0] = vk.v[k][n];
            w[k][1] = vk.v[k][N + n];
            w[k][2] = d == 3 ? vk.v[k][2 * N + n] : 0.f;
        }
        int idx = 0;
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[idx++] += u[0] * w[k][0] + u[1] * w[k][1] + u[2] * w[k][2];
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int j = i; j < NS; ++j) acc[idx++] += w[i][0] * w[j][0] + w[i][1] * w[j][1] + w[i][2] * w[j][2];
        acc[idx++] += u[0];
#pragma unroll
        for (int k = 0; k < NS; ++k) acc[idx++] += w[k][0];
    }
    __shared__ float sh[4][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        float a = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[wid][v] = a;
    }
    __syncthreads();
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        const float s = (sh[0][v] + sh[1][v]) + (sh[2][v] + sh[3][v]);
        if (v < NS + NG) part[(size_t)blk * (NS + NG) + v] = s;
        else plane_part[((size_t)zc * p.ny + y) * (1 + NS) + (v - NS - NG)] = s;
    }
}

// ------------------------------------------- LRS history matvec, normals --
// Runs on a side branch of the step (it needs only the previous step's
// histories and the step counter), so its latency hides behind the field
// kernels.  Blocks 0..nblk_lrs-1: partial sums of x_r C[r][:] over the rows of
// C whose inputs are known before the current QoIs: the histories
// q^{n-1..n-h} and q^{n-1*..n-h*} (scaled by sigma_ref) and the bias 1
// (Eq. LRS); the q^{n*} block is added in the solve.  A block first forms its
// rows' inputs x_r in shared memory (one division each, as in the model),
// then thread (j, k) accumulates rows j, j + per, ... of column k, so a warp
// reads consecutive elements of C.  The last block draws the step's normals
// (the LRS noise or the gamma draws).
__global__ void __launch_bounds__(256) lrs_pre_kernel(Params p, Layout L, int nb) {
    const int nq = p.n_q;
    const long long step = L.st->step;
    if (blockIdx.x == (unsigned)nb) {
        const int stream = p.to_mode == LBM_TO_GAMMA ? kStreamGamma : kStreamLrs;
        if (threadIdx.x < (unsigned)nq) L.znorm[threadIdx.x] = philox_normal(p.seed, p.member, step, stream, threadIdx.x);
        return;
    }
    const int h = p.h;
    const int rows = (2 * h + 1) * nq + 1;
    const int r0 = blockIdx.x * p.lrs_rows_per_blk;
    const int r1 = min(rows, r0 + p.lrs_rows_per_blk);
    const int posm = (int)(L.st->hist_pos % h);
    __shared__ double xs[kLrsRowsPerBlk];
    __shared__ double sh[256];
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double xr = 0.0;
        if (r < h * nq || (r >= (h + 1) * nq && r < rows - 1)) {
            const bool corrected = r < h * nq;
            const int rr = corrected ? r : r - (h + 1) * nq;
            const int kk = rr / nq + 1, i = rr - (kk - 1) * nq;
            int slot = posm - kk;
            if (slot < 0) slot += h;
            const double sg = L.lrs_sigma[i];
            const double qv = corrected ? L.qh[(size_t)slot * nq + i] : L.qsh[(size_t)slot * nq + i];
            xr = sg > 0.0 ? qv / sg : 0.0;  // sigma <= 0: not yet set, the histories are zero
        } else if (r == rows - 1) {
            xr = 1.0;
        }  // rows of the q^{n*} block: added in the solve
        xs[r - r0] = xr;
    }
    __syncthreads();
    const int per = blockDim.x / nq;
    const int j = threadIdx.x / nq, k = threadIdx.x - j * nq;
    double acc = 0.0;
    if (j < per)
        for (int r = r0 + j; r < r1; r += per) acc = fma(xs[r - r0], L.lrs_C[(size_t)r * nq + k], acc);
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < (unsigned)nq) {
        double s = 0.0;
        for (int jj = 0; jj < per; ++jj) s += sh[jj * nq + threadIdx.x];
        L.lrs_part[(size_t)blockIdx.x * nq + threadIdx.x] = s;
    }
}

// ------------------------------------------------------------- solve --
// One block: sum the partials, assemble q^{n*} and the Gram matrix, evaluate
// the coefficient source, factor G = X^-1 D X^-T (LDL^T, FP64), and produce
// beta = G^-1 dQ (dv_SGS = sum_k beta_k V_k equals sum_i gamma_i O_i with c_ij
// and gamma_i of Sec. 4.2-4.3), gamma_i = dQ_i (G^-1)_ii.  Then write the QoI
// block row, push the LRS histories, add the mean profile and advance the step
// counter.
//
// Double-precision operations issue slowly on this GPU and this kernel is on
// the critical path of every step, so its FP64 work is arranged as short
// parallel chains: sums of FP32 partials are compensated single-precision
// sums widened once, the factorisation is right-looking with one reciprocal
// per pivot, and the triangular products run one row/column per lane.
__global__ void __launch_bounds__(256) solve_kernel(Params p, Layout L) {
    const int ns = p.n_s, nmp = p.n_mp, nq = p.n_q;
    const int ng = ns * (ns + 1) / 2;
    const int npart = ns + ng;
    __shared__ double red[kMaxQoi + kMaxQoi * (kMaxQoi + 1) / 2];
    __shared__ double A[kMaxQoi][kMaxQoi + 1];   // G, overwritten by the factorisation
    __shared__ double Lc[kMaxQoi][kMaxQoi + 1];  // unit lower factor
    __shared__ double X[kMaxQoi][kMaxQoi + 1];   // its inverse
    __shared__ double invD[kMaxQoi];
    __shared__ double q[kMaxQoi], dq[kMaxQoi], beta[kMaxQoi], z[kMaxQoi], hpart[kMaxQoi], qnew[kMaxQoi];
    __shared__ double xq[kMaxQoi], yv[kMaxQoi];
    __shared__ double wP[kMaxQoi][kMaxQoi + 1];  // sum_y w_j(y) P_k(y), k = 0 (v_x), 1..ns (V_k,x)
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const long long step = L.st->step;
    const bool lrs = p.to_mode == LBM_TO_LRS;

    // 1. totals of the block partials (one warp per value) and the LRS
    //    history partials; plane sums P_k(y) over the z chunks (one per thread)
    for (int v = wid; v < npart; v += nw) {
        const double a = df_warp_sum(L.part + v, p.nblk_red, (size_t)npart, lane);
        if (lane == 0) red[v] = a;
    }
    if (lrs)
        for (int k = wid; k < nq; k += nw) {
            double a = 0.0;
            for (int b = lane; b < p.nblk_lrs; b += 32) a += L.lrs_part[(size_t)b * nq + k];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) hpart[k] = a;
        }
    const int np1 = 1 + ns;
    for (int e = tid; e < p.ny * np1; e += blockDim.x) {
        DF a = {0.f, 0.f};
        for (int zc = 0; zc < p.nzc; ++zc) a = df_add(a, L.plane_part[((size_t)zc * p.ny) * np1 + e]);
        L.plane_sum[e] = (double)a.hi + (double)a.lo;
    }
    __syncthreads();
    // 2. mean-profile couplings sum_y w_j(y) P_k(y): one warp per (j, k), lanes over y
    for (int e = wid; e < nmp * np1; e += nw) {
        const int j = e / np1, k = e - j * np1;
        double a = 0.0;
        for (int y = lane; y < p.ny; y += 32) a = fma(L.w_mp[(size_t)j * p.ny + y], L.plane_sum[(size_t)y * np1 + k], a);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) wP[j][k] = a;
    }
    __syncthreads();
    // 3. q^{n*}, G, the normals, reference scales (warp 0, lane i = QoI i)
    if (wid == 0) {
        const int i = lane;
        double gdiag = 0.0;
        if (i < nq) {
            q[i] = i < ns ? 0.5 * red[i] : wP[i - ns][0];
            for (int j = 0; j < nq; ++j) {
                double gij;
                if (i < ns && j < ns) {
                    const int a = min(i, j), b = max(i, j);
                    gij = red[ns + a * ns - a * (a - 1) / 2 + (b - a)];
                } else if (i >= ns && j >= ns) {
                    gij = L.g_mpmp[(size_t)(i - ns) * nmp + (j - ns)];
                } else if (i >= ns) {
                    gij = wP[i - ns][1 + j];
                } else {
                    gij = wP[j - ns][1 + i];
                }
                A[i][j] = gij;
                if (j == i) gdiag = gij;
            }
            z[i] = (lrs || p.to_mode == LBM_TO_GAMMA) ? L.znorm[i] : 0.0;
            if (lrs) {
                // a reference scale <= 0 is taken from this step's predictor QoI
                double sg = L.lrs_sigma[i];
                if (!(sg > 0.0)) {
                    sg = fabs(q[i]) > 0.0 ? fabs(q[i]) : 1.0;
                    L.lrs_sigma[i] = sg;
                }
                xq[i] = q[i] / sg;
            }
        }
        // 4. LDL^T with the pivot test d_k > 1e-14 max_i G_ii (the Schur
        //    complements are the Cholesky pivots of Sec. 4.3's singular test)
        double dmax = gdiag;
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        int sing = !(dmax > 0.0);
        __syncwarp();
        for (int k = 0; k < nq && !sing; ++k) {
            const double dk = A[k][k];
            if (!(dk > 1e-14 * dmax)) { sing = 1; break; }
            const double inv = 1.0 / dk;
            if (i == k) { invD[k] = inv; Lc[k][k] = 1.0; }
            if (i > k && i < nq) Lc[i][k] = A[i][k] * inv;
            __syncwarp();
            // trailing update A_ij -= L_ik A_jk (k < j <= i), lanes over i
            if (i > k && i < nq) {
                const double lik = Lc[i][k];
                for (int j = k + 1; j <= i; ++j) A[i][j] = fma(-lik, A[j][k], A[i][j]);
            }
            __syncwarp();
        }
        // X = Lc^-1 (unit lower): lane c owns column c, rows in order
        if (!sing && i < nq) {
            for (int r = 0; r < nq; ++r) {
                double a = r == i ? 1.0 : 0.0;
                if (r > i)
                    for (int m = i; m < r; ++m) a = fma(-Lc[r][m], X[m][i], a);
                X[r][i] = a;
            }
        }
        __syncwarp();
        // 5. coefficient source -> dQ, gamma; G^-1 = X^T D^-1 X
        double d = 0.0, g = 0.0;
        if (i < nq) {
            double ginv_ii = 0.0;
            if (!sing)
                for (int r = i; r < nq; ++r) ginv_ii = fma(X[r][i] * X[r][i], invD[r], ginv_ii);
            if (lrs && step < p.spinup) {
                // spin-up: nudged to the reference, which enters the history
                const long long row = step < p.track_len ? step : p.track_len - 1;
                const double qref = L.track[(size_t)row * nq + i];
                d = qref - q[i];
                qnew[i] = qref;
                g = sing ? 0.0 : d * ginv_ii;
            } else if (lrs) {
                double qh = hpart[i] + L.lrs_mu[i];
                for (int j = 0; j < nq; ++j)
                    qh += xq[j] * L.lrs_C[((size_t)p.h * nq + j) * nq + i] + L.lrs_L[(size_t)i * nq + j] * z[j];
                const double qn = L.lrs_sigma[i] * qh;
                d = qn - q[i];
                qnew[i] = qn;  // corrected QoI for the history
                g = sing ? 0.0 : d * ginv_ii;
            } else if (p.to_mode == LBM_TO_GAMMA) {
                if (!sing) {
                    g = p.gamma_std * z[i];
                    d = g / ginv_ii;
                }
            } else if (p.to_mode == LBM_TO_TRACK) {
                const long long row = step < p.track_len ? step : p.track_len - 1;
                d = L.track[(size_t)row * nq + i] - q[i];
                g = sing ? 0.0 : d * ginv_ii;
            }
            dq[i] = d;
        }
        __syncwarp();
        // beta = X^T D^-1 X dQ: lane r forms (X dQ)_r / D_r, then lane c sums column c
        const bool skip = sing || p.to_mode == LBM_TO_OBSERVE;
        if (i < nq) {
            double a = 0.0;
            if (!skip)
                for (int m = 0; m <= i; ++m) a = fma(X[i][m], dq[m], a);
            yv[i] = skip ? 0.0 : a * invD[i];
        }
        __syncwarp();
        if (i < nq) {
            double a = 0.0;
            if (!skip)
                for (int r = i; r < nq; ++r) a = fma(X[r][i], yv[r], a);
            beta[i] = a;
            L.beta[i] = a;
            // QoI block row
            const long long rc = L.st->ring_count;
            double* row = L.ring + (size_t)(rc % p.ring_cap) * p.row_len;
            if (i == 0) row[0] = (double)step;
            row[1 + i] = q[i];
            row[1 + nq + i] = d;
            row[1 + 2 * nq + i] = g;
            if (i == 0) {
                unsigned fl = sing ? LBM_FLAG_SINGULAR : 0u;
                if (L.st->status & 1u) fl |= LBM_FLAG_UNSTABLE;
                row[1 + 3 * nq] = (double)fl;
            }
            if (lrs && p.h > 0) {
                const long long slot = L.st->hist_pos % p.h;
                L.qh[slot * nq + i] = qnew[i];
                L.qsh[slot * nq + i] = q[i];
            }
        }
        __syncwarp();
        if (lane == 0) {
            L.st->ring_count += 1;
            if (lrs && p.h > 0) L.st->hist_pos += 1;
        }
    }
    __syncthreads();
    // 6. mean profile of the corrected velocity: P_v + sum_k beta_k P_k + nx nz sum_j beta_mp_j w_j
    const double area = (double)p.nx * (double)p.nz;
    for (int y = tid; y < p.ny; y += blockDim.x) {
        double a = L.plane_sum[(size_t)y * np1];
        for (int k = 0; k < ns; ++k) a = fma(beta[k], L.plane_sum[(size_t)y * np1 + 1 + k], a);
        for (int j = 0; j < nmp; ++j) a = fma(area * beta[ns + j], L.w_mp[(size_t)j * p.ny + y], a);
        L.profile[y] += a / area;
    }
    if (tid == 0) {
        L.st->prof_steps += 1;
        L.st->step = step + 1;
    }
}

// ------------------------------------------------------------ launchers --
static inline unsigned gridn(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_to_curl(const Params& p, const Layout& L, cudaStream_t s) {
    curl_kernel<<<gridn(p.n, 256), 256, 0, s>>>(p, L.x6);
    return cudaGetLastError();
}
cudaError_t launch_pass(const Params& p, const float* in, float* out, int ncomp, int axis, const Taps& t, float scale,
                        int accumulate, cudaStream_t s) {
    const cudaError_t e = launch_pass_fast(p, in, out, ncomp, axis, t, scale, accumulate, s);
    if (e != cudaErrorNotSupported) return e;
    pass_kernel<<<gridn(p.n, 256), 256, 0, s>>>(p, in, out, ncomp, axis, t, scale, accumulate);
    return cudaGetLastError();
}
cudaError_t launch_band_mask(const Params& p, const float2* in, float2* out, int ncomp, int lo, int hi,
                             cudaStream_t s) {
    const long long n = (long long)p.ny * (p.nx / 2 + 1) * ncomp;
    band_mask_kernel<<<gridn(n, 256), 256, 0, s>>>(p, in, out, ncomp, lo, hi);
    return cudaGetLastError();
}
cudaError_t launch_sens_curl(const Params& p, const float* w, float* out, cudaStream_t s) {
    sens_curl_kernel<<<gridn(p.n, 256), 256, 0, s>>>(p, w, out);
    return cudaGetLastError();
}
cudaError_t launch_reduce(const Params& p, const Layout& L, const float* const* vk, cudaStream_t s) {
    RedPtrs r;
    for (int k = 0; k < kMaxQoi; ++k) r.v[k] = k < p.n_s ? vk[k] : nullptr;
    dim3 grid(p.ny, p.nzc);
    switch (p.n_s) {
        case 1: reduce_kernel<1><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        case 2: reduce_kernel<2><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        case 3: reduce_kernel<3><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        case 4: reduce_kernel<4><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        case 5: reduce_kernel<5><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        case 6: reduce_kernel<6><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        case 7: reduce_kernel<7><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        case 8: reduce_kernel<8><<<grid, 128, 0, s>>>(p, L.vps, r, L.part, L.plane_part); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
cudaError_t launch_lrs_pre(const Params& p, const Layout& L, cudaStream_t s) {
    const int nb = p.to_mode == LBM_TO_LRS ? p.nblk_lrs : 0;
    lrs_pre_kernel<<<nb + 1, 256, 0, s>>>(p, L, nb);
    return cudaGetLastError();
}
cudaError_t launch_solve(const Params& p, const Layout& L, cudaStream_t s) {
    solve_kernel<<<1, 256, 0, s>>>(p, L);
    return cudaGetLastError();
}

}  // namespace lbm
