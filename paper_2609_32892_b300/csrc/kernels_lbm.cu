// Stream-collide, SGS apply and state conversion kernels (D2Q9 / D3Q19).
//
// Populations are stored shifted, g_i = f_i - w_i, in FP32, FP16 or BF16, as
// [Q][nz][ny][nx] arrays; all arithmetic is FP32.  Writing the equilibrium and
// the forcing terms as deviations (delta rho = sum g, rho u = sum c g, since
// sum w = 1 and sum w c = 0) keeps the small velocity-carrying part of each
// population at full relative precision.
#include "batch.cuh"
#include "lbm_common.cuh"

namespace lbm {

// ---------------------------------------------------------------- lattice --
// Velocity sets in the library's population order (see lbm.h); constexpr so
// that fully unrolled loops fold every c_i and w_i into immediates.
template <int DIM> struct Lat;

template <> struct Lat<2> {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[i];
    }
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
    }
};

template <> struct Lat<3> {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
        return t[i];
    }
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 1.0f / 3.0f : (i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
    }
};

// ---------------------------------------------------------------- storage --
template <typename T> __device__ __forceinline__ float ldg_(const T* p);
template <> __device__ __forceinline__ float ldg_<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldg_<__half>(const __half* p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float ldg_<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}
template <typename T> __device__ __forceinline__ float ld_(const T* p);
template <> __device__ __forceinline__ float ld_<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_<__half>(const __half* p) { return __half2float(*p); }
template <> __device__ __forceinline__ float ld_<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <typename T> __device__ __forceinline__ void st_(T* p, float v);
template <> __device__ __forceinline__ void st_<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void st_<__half>(__half* p, float v) { *p = __float2half_rn(v); }
template <> __device__ __forceinline__ void st_<__nv_bfloat16>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}

__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// -------------------------------------------------------------- pull + moments
// Pull-stream the populations arriving at node (x, y, z) (Eq. LES-3 of the
// previous step): g_i(x) = g^p_i(x - c_i), or, if x - c_i is a solid row,
// halfway bounce-back g_i(x) = g^p_{opp(i)}(x).
template <int DIM, typename T>
__device__ __forceinline__ void pull(const Params& p, const T* __restrict__ src, int x, int y, int z, int n,
                                     float* g) {
    using LT = Lat<DIM>;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int N = (int)p.n;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    const int ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
    const int zm = DIM == 3 ? wrap(z - 1, nz) : 0, zp = DIM == 3 ? wrap(z + 1, nz) : 0;
    const bool wall_lo = p.walls && (y == 1);        // source row y-1 solid
    const bool wall_hi = p.walls && (y == ny - 2);   // source row y+1 solid
    // node offsets within one population array fit in 32 bits (6 N < 2^31);
    // the population arrays are stepped through by pointer (Q N may not)
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const int cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
        const bool bb = (cy == 1 && wall_lo) || (cy == -1 && wall_hi);
        if (bb) {
            g[i] = ldg_<T>(src + (size_t)LT::opp(i) * N + n);
        } else {
            const int xs = cx == 0 ? x : (cx > 0 ? xm : xp);
            const int ys = cy == 0 ? y : (cy > 0 ? ym : yp);
            const int zs = cz == 0 ? z : (cz > 0 ? zm : zp);
            g[i] = ldg_<T>(src + (size_t)i * N + (unsigned)((zs * ny + ys) * nx + xs));
        }
    }
}

struct Macro {
    float drho, rho, jx, jy, jz;   // deviation density, density, momentum sum c g
    float fx, fy, fz;              // force density
    float ux, uy, uz;              // equilibrium velocity (EDM: j/rho, Guo: (j + F/2)/rho)
};

// ACC: u = (rho u)/rho by IEEE division (FP32 storage, where the collision's
// rounding sets the error); otherwise by one reciprocal (16-bit storage, where
// storage rounding dominates and the kernel is arithmetic bound).
template <int DIM, bool ACC = true>
__device__ __forceinline__ Macro macros_of(const Params& p, const float* g, const float* kolmo, int y) {
    using LT = Lat<DIM>;
    Macro m;
    float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        dr += g[i];
        if (LT::cx(i)) jx += LT::cx(i) * g[i];
        if (LT::cy(i)) jy += LT::cy(i) * g[i];
        if (DIM == 3 && LT::cz(i)) jz += LT::cz(i) * g[i];
    }
    m.drho = dr;
    m.rho = 1.0f + dr;
    m.jx = jx; m.jy = jy; m.jz = jz;
    // F = F_body + A sin(2 pi k y / ny) e_x - alpha rho u
    m.fx = p.body[0] + kolmo[y] - p.kolmo_drag * jx;
    m.fy = p.body[1] - p.kolmo_drag * jy;
    m.fz = DIM == 3 ? p.body[2] - p.kolmo_drag * jz : 0.f;
    if (ACC) {
        // quotient from the reciprocal plus one Newton correction of the
        // residual (Markstein 1990): q = n r, q += (n - q rho) r, as accurate
        // as a correctly rounded division for these operands at a third of the cost
        const float inv = 1.0f / m.rho;
        const float nx_ = p.forcing == LBM_FORCING_GUO ? jx + 0.5f * m.fx : jx;
        const float ny_ = p.forcing == LBM_FORCING_GUO ? jy + 0.5f * m.fy : jy;
        const float nz_ = p.forcing == LBM_FORCING_GUO ? jz + 0.5f * m.fz : jz;
        float qx = nx_ * inv, qy = ny_ * inv, qz = nz_ * inv;
        qx = fmaf(fmaf(-qx, m.rho, nx_), inv, qx);
        qy = fmaf(fmaf(-qy, m.rho, ny_), inv, qy);
        qz = fmaf(fmaf(-qz, m.rho, nz_), inv, qz);
        m.ux = qx;
        m.uy = qy;
        m.uz = qz;
    } else {
        const float inv = 1.0f / m.rho;
        if (p.forcing == LBM_FORCING_GUO) {
            m.ux = (jx + 0.5f * m.fx) * inv;
            m.uy = (jy + 0.5f * m.fy) * inv;
            m.uz = (jz + 0.5f * m.fz) * inv;
        } else {
            m.ux = jx * inv;
            m.uy = jy * inv;
            m.uz = jz * inv;
        }
    }
    return m;
}

// The predictor velocity of the TO phase (Sec. 4 predictor-corrector):
// BGK relaxation conserves mass and momentum and the body force adds F, so
// v^{p*} = sum_i c_i f^{p*}_i / rho = (rho u + F)/rho under both forcing
// schemes.  It follows from the pulled moments alone, whatever tau_eff the
// substrate gives the node, so it can be formed before the collision.
__device__ __forceinline__ void predictor_velocity(const Macro& m, float& vx, float& vy, float& vz) {
    const float inv = 1.0f / m.rho;
    vx = (m.jx + m.fx) * inv;
    vy = (m.jy + m.fy) * inv;
    vz = (m.jz + m.fz) * inv;
}

// ------------------------------------------------------------------ kernels --
// Predictor pass: pull the populations of a node and write the predictor
// velocity v^{p*} (WV, the input of the TO phase, DIM components) and/or the
// post-stream velocity u (WN, the input of the WALE gradients, 3 components).
// Solid rows get zero velocity.
template <int DIM, typename T, bool WV, bool WN>
__device__ __forceinline__ void predict_kernel_body(const VB& vb, const Params& p, const T* __restrict__ src,
                                                    float* __restrict__ vps, float* __restrict__ vn,
                                                    const float* __restrict__ kolmo) {
    const int n = vb.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n;
    const int x = n % p.nx;
    const int t = n / p.nx;
    const int y = t % p.ny;
    const int z = t / p.ny;
    float vx = 0.f, vy = 0.f, vz = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
    if (!(p.walls && (y == 0 || y == p.ny - 1))) {
        float g[Lat<DIM>::Q];
        pull<DIM, T>(p, src, x, y, z, n, g);
        const Macro m = macros_of<DIM>(p, g, kolmo, y);
        predictor_velocity(m, vx, vy, vz);
        ux = m.ux; uy = m.uy; uz = m.uz;
    }
    if (WV) {
        vps[n] = vx;
        vps[(size_t)N + n] = vy;
        if (DIM == 3) vps[(size_t)2 * N + n] = vz;
    }
    if (WN) {
        vn[n] = ux;
        vn[(size_t)N + n] = uy;
        vn[(size_t)2 * N + n] = uz;
    }
}
template <int DIM, typename T, bool WV, bool WN>
struct predict_kernel_op {
    static constexpr int NT = 256, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        predict_kernel_body<DIM, T, WV, WN>(vb, b...);
    }
};
template <int DIM, typename T, bool WV, bool WN>
__global__ void __launch_bounds__(256) predict_kernel(Params p, const T* __restrict__ src, float* __restrict__ vps,
                                                      float* __restrict__ vn, const float* __restrict__ kolmo) {
    predict_kernel_body<DIM, T, WV, WN>(vb_hw(), p, src, vps, vn, kolmo);
}

// WALE eddy viscosity from the post-stream velocity field (Sec. 5.2): g_ij =
// d_j v_i by central differences (zero velocity on solid rows), then
// nu_t = C_w^2 (Sd:Sd)^{3/2} / ((S:S)^{5/2} + (Sd:Sd)^{5/4}), 0 if that
// denominator is below 1e-30.
template <int DIM>
__device__ __forceinline__ float wale_nut(const Params& p, const float* __restrict__ vn, int x, int y, int z) {
    const int N = (int)p.n, nx = p.nx, ny = p.ny, nz = p.nz;
    float gm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) gm[a][b] = 0.f;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    const int ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
    // 32-bit node offsets (6 N < 2^31)
    const unsigned row = (unsigned)((z * ny + y) * nx);
    const unsigned iyp = (unsigned)((z * ny + yp) * nx + x), iym = (unsigned)((z * ny + ym) * nx + x);
    const int zm = DIM == 3 ? wrap(z - 1, nz) : 0, zp = DIM == 3 ? wrap(z + 1, nz) : 0;
    const unsigned izp = (unsigned)((zp * ny + y) * nx + x), izm = (unsigned)((zm * ny + y) * nx + x);
#pragma unroll
    for (int i = 0; i < (DIM == 3 ? 3 : 2); ++i) {
        const float* v = vn + (size_t)i * N;
        gm[i][0] = 0.5f * (v[row + xp] - v[row + xm]);
        gm[i][1] = 0.5f * (v[iyp] - v[iym]);
        if (DIM == 3) gm[i][2] = 0.5f * (v[izp] - v[izm]);
    }
    float g2[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) g2[a][b] = gm[a][0] * gm[0][b] + gm[a][1] * gm[1][b] + gm[a][2] * gm[2][b];
    const float tr = g2[0][0] + g2[1][1] + g2[2][2];
    float ss = 0.f, sdsd = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float s = 0.5f * (gm[a][b] + gm[b][a]);
            float sd = 0.5f * (g2[a][b] + g2[b][a]);
            if (a == b) sd -= tr * (1.0f / 3.0f);
            ss += s * s;
            sdsd += sd * sd;
        }
    const float den = ss * ss * sqrtf(ss) + sdsd * sqrtf(sqrtf(sdsd));
    if (!(den >= 1e-30f)) return 0.f;
    return p.c_wale2 * sdsd * sqrtf(sdsd) / den;
}

// The collision of one node from its pulled populations g (in place):
// moments, substrate tau_eff, BGK (Eq. LES-1), the body force and, with CORR,
// the step's SGS increment dv (Eq. LES-2).  Under EDM the force and the SGS
// increment form one equilibrium difference, Eq. LES-2's single-difference
// form f^a + f^eq(rho, u + F/rho + dv) - f^eq(rho, u) (the predictor form
// f^{p*} + f^eq(v* + dv) - f^eq(v*), v* = u + F/rho, telescopes to it); under
// Guo's scheme the increment follows the forcing as its own difference.
template <int DIM>
__device__ __forceinline__ void sgs_correct(float* g, float r, float ux, float uy, float uz, float dx, float dy,
                                            float dz);

template <int DIM, int SUB, bool ACC, bool CORR>
__device__ __forceinline__ void collide_node(const Params& p, float* g, int x, int y, int z,
                                             const float* __restrict__ vn, const float* __restrict__ kolmo,
                                             DevState* st, float dvx, float dvy, float dvz) {
    using LT = Lat<DIM>;
    const Macro m = macros_of<DIM, ACC>(p, g, kolmo, y);
    const float ux = m.ux, uy = m.uy, uz = m.uz;
    const float uu = ux * ux + uy * uy + uz * uz;
    if (!(m.rho > 0.f) || !(uu <= (1.0f / 3.0f))) atomicOr(&st->status, 1u);

    // equilibrium deviations g^eq_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 uu)).
    // FP32 storage: one expression per direction (measured most accurate against
    // the FP64 reference); 16-bit storage: per opposite pair (i, opp i), the
    // even part shared and the odd part 3 w rho cu flipping sign (fewer
    // operations for the arithmetic-bound 16-bit kernel).
    float geq[LT::Q];
    if (ACC) {
#pragma unroll
        for (int i = 0; i < LT::Q; ++i) {
            const float cu = LT::cx(i) * ux + LT::cy(i) * uy + LT::cz(i) * uz;
            geq[i] = LT::w(i) * (m.drho + m.rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
        }
    } else {
        geq[0] = LT::w(0) * (m.drho - 1.5f * m.rho * uu);
#pragma unroll
        for (int i = 1; i < LT::Q; ++i) {
            if (LT::opp(i) < i) continue;
            const float cu = LT::cx(i) * ux + LT::cy(i) * uy + LT::cz(i) * uz;
            const float ev = LT::w(i) * (m.drho + m.rho * (4.5f * cu * cu - 1.5f * uu));
            const float od = LT::w(i) * m.rho * 3.0f * cu;
            geq[i] = ev + od;
            geq[LT::opp(i)] = ev - od;
        }
    }
    // Without a substrate 1/tau and 1 - 1/(2 tau) come rounded once from
    // double: the viscosity depends on (1/omega - 1/2) and Guo's prefactor is
    // a small difference, so FP32 recomputation would bias both by ~1e-6.
    float tau = p.tau;
    float om = p.omega0;
    float pre = p.guo_pre0;
    if (SUB == LBM_SUBSTRATE_SMAG) {
        // Pi^neq_ab = sum_i c_ia c_ib (f_i - f^eq_i); tau_eff closed form (Sec. 5.1)
        float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
        for (int i = 0; i < LT::Q; ++i) {
            const float d = g[i] - geq[i];
            const int cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
            if (cx) pxx += d;
            if (cy) pyy += d;
            if (cz) pzz += d;
            if (cx * cy) pxy += (cx * cy) * d;
            if (cx * cz) pxz += (cx * cz) * d;
            if (cy * cz) pyz += (cy * cz) * d;
        }
        const float pn = sqrtf(2.0f * (pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz)));
        tau = 0.5f * (p.tau + sqrtf(p.tau * p.tau + 18.0f * p.c_smag2 * pn / m.rho));
    } else if (SUB == LBM_SUBSTRATE_WALE) {
        tau = p.tau + 3.0f * wale_nut<DIM>(p, vn, x, y, z);
    }
    if (SUB != LBM_SUBSTRATE_NONE) {
        om = 1.0f / tau;
        pre = (tau - 0.5f) * om;  // tau - 1/2 is exact in FP32 for tau in [1/2, 1]
    }

    // body-force terms, again per opposite pair (even part shared, odd part flips)
    const float fx = m.fx, fy = m.fy, fz = m.fz;
    if (p.forcing == LBM_FORCING_GUO) {
        // S_i = w (1 - 1/(2 tau)) [3 (c - u).F + 9 (c.u)(c.F)]
        const float uf = ux * fx + uy * fy + uz * fz;
        g[0] = g[0] + (geq[0] - g[0]) * om - LT::w(0) * pre * 3.0f * uf;
#pragma unroll
        for (int i = 1; i < LT::Q; ++i) {
            if (LT::opp(i) < i) continue;
            const int cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cf = cx * fx + cy * fy + cz * fz;
            const float ev = LT::w(i) * pre * (9.0f * cu * cf - 3.0f * uf);
            const float od = LT::w(i) * pre * 3.0f * cf;
            const int j = LT::opp(i);
            g[i] = g[i] + (geq[i] - g[i]) * om + (ev + od);
            g[j] = g[j] + (geq[j] - g[j]) * om + (ev - od);
        }
    } else {
        // EDM: S_i = w rho [3 c.d + 4.5 (c.d)(2 c.u + c.d) - 1.5 d.(2u + d)], d = F/rho
        const float inv = 1.0f / m.rho;
        float dx = fx * inv, dy = fy * inv, dz = fz * inv;
        if (CORR) {
            dx += dvx;
            dy += dvy;
            dz += dvz;
        }
        const float du = dx * (2.0f * ux + dx) + dy * (2.0f * uy + dy) + dz * (2.0f * uz + dz);
        g[0] = g[0] + (geq[0] - g[0]) * om - LT::w(0) * m.rho * 1.5f * du;
#pragma unroll
        for (int i = 1; i < LT::Q; ++i) {
            if (LT::opp(i) < i) continue;
            const int cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cd = cx * dx + cy * dy + cz * dz;
            const float ev = LT::w(i) * m.rho * (4.5f * cd * (2.0f * cu + cd) - 1.5f * du);
            const float od = LT::w(i) * m.rho * 3.0f * cd;
            const int j = LT::opp(i);
            g[i] = g[i] + (geq[i] - g[i]) * om + (ev + od);
            g[j] = g[j] + (geq[j] - g[j]) * om + (ev - od);
        }
    }
    if (CORR && p.forcing == LBM_FORCING_GUO) {
        float vx, vy, vz;
        predictor_velocity(m, vx, vy, vz);
        sgs_correct<DIM>(g, m.rho, vx, vy, vz, dvx, dvy, dvz);
    }
}

// SGS velocity increment of a node: dv = sum_k beta_k V_k + (sum_j beta_j
// w_j(y)) e_x (the orthogonal patterns folded into one combination of the
// sensitivities, beta = G^-1 dQ; the band term per row from the solve).
struct VPtrs {
    const float* v[kMaxQoi];
};
constexpr int kMaxScaleQoi = 8;  // lbm_create allows at most 8 scale-aware QoIs

template <int DIM>
__device__ __forceinline__ void sgs_increment(const Params& p, const VPtrs& vk, const float* __restrict__ betaf,
                                              const float* __restrict__ mprow, size_t n, int y, float& dx,
                                              float& dy, float& dz) {
    const size_t N = (size_t)p.n;
    dx = 0.f;
    dy = 0.f;
    dz = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxScaleQoi; ++k) {
        if (k < p.n_s) {
            const float b = betaf[k];
            const float* v = vk.v[k];
            dx += b * __ldg(v + n);
            dy += b * __ldg(v + N + n);
            if (DIM == 3) dz += b * __ldg(v + 2 * N + n);
        }
    }
    dx += mprow[y];
}

// Eq. LES-2 corrector on the predictor populations of a node held in
// registers: g^p = g^{p*} + f^eq(rho, v* + dv) - f^eq(rho, v*), written out
// as w_i rho [3 c.d + 4.5 (c.d)(2 c.v* + c.d) - 1.5 d.(2 v* + d)].
template <int DIM>
__device__ __forceinline__ void sgs_correct(float* g, float r, float ux, float uy, float uz, float dx, float dy,
                                            float dz) {
    using LT = Lat<DIM>;
    const float du = dx * (2.0f * ux + dx) + dy * (2.0f * uy + dy) + dz * (2.0f * uz + dz);
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const int cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
        const float cu = cx * ux + cy * uy + cz * uz;
        const float cd = cx * dx + cy * dy + cz * dz;
        g[i] += LT::w(i) * r * (3.0f * cd + 4.5f * cd * (2.0f * cu + cd) - 1.5f * du);
    }
}

// One thread per node: pull, collide_node and, with CORR, the SGS corrector
// of the step (Eq. LES-2) before the store: the predictor populations never
// leave registers.
//
// 3-D FP32 launches collide4_kernel: four 256-thread blocks per SM (64
// registers; the WALE corrector form takes 80 otherwise, three blocks).  The
// kernel waits on its population, sensitivity and velocity loads, and the
// fourth block hides more of that latency than the few spilled bytes cost
// (1.17 -> 1.15 ms at 480 x 200 x 240).  16-bit storage and 2-D keep
// collide_kernel and the compiler's register choice (the 16-bit forms are
// arithmetic bound and would spill more under the cap).
template <int DIM, typename T>
constexpr int collide_minb() {
    return DIM == 3 && sizeof(T) == 4 ? 4 : 1;
}
template <int DIM, typename T, int SUB, bool CORR>
__device__ __forceinline__ void collide_kernel_body(const VB& vb, const Params& p, const T* __restrict__ src,
                                                    T* __restrict__ dst, const float* __restrict__ vn,
                                                    const float* __restrict__ kolmo, DevState* st, VPtrs vk,
                                                    const float* __restrict__ betaf,
                                                    const float* __restrict__ mprow) {
    using LT = Lat<DIM>;
    const int n = vb.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n;
    const int x = n % p.nx;
    const int t = n / p.nx;
    const int y = t % p.ny;
    const int z = t / p.ny;
    if (p.walls && (y == 0 || y == p.ny - 1)) return;
    float g[LT::Q];
    pull<DIM, T>(p, src, x, y, z, n, g);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    if (CORR) sgs_increment<DIM>(p, vk, betaf, mprow, (size_t)n, y, dx, dy, dz);
    collide_node<DIM, SUB, (sizeof(T) == 4), CORR>(p, g, x, y, z, vn, kolmo, st, dx, dy, dz);
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) st_<T>(dst + (size_t)i * N + n, g[i]);
}
template <int DIM, typename T, int SUB, bool CORR>
struct collide_kernel_op {
    static constexpr int NT = 256, MINB = collide_minb<DIM, T>();
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        collide_kernel_body<DIM, T, SUB, CORR>(vb, b...);
    }
};
template <int DIM, typename T, int SUB, bool CORR>
__global__ void __launch_bounds__(256) collide_kernel(Params p, const T* __restrict__ src, T* __restrict__ dst,
                                                      const float* __restrict__ vn, const float* __restrict__ kolmo,
                                                      DevState* st, VPtrs vk, const float* __restrict__ betaf,
                                                      const float* __restrict__ mprow) {
    collide_kernel_body<DIM, T, SUB, CORR>(vb_hw(), p, src, dst, vn, kolmo, st, vk, betaf, mprow);
}
template <int DIM, typename T, int SUB, bool CORR>
__global__ void __launch_bounds__(256, 4) collide4_kernel(Params p, const T* __restrict__ src, T* __restrict__ dst,
                                                          const float* __restrict__ vn, const float* __restrict__ kolmo,
                                                          DevState* st, VPtrs vk, const float* __restrict__ betaf,
                                                          const float* __restrict__ mprow) {
    collide_kernel_body<DIM, T, SUB, CORR>(vb_hw(), p, src, dst, vn, kolmo, st, vk, betaf, mprow);
}

// ---- two nodes per thread (nx even): aligned 2-element population loads ----
template <typename T> struct Vec2;
template <> struct Vec2<float> {
    using V = float2;
    static __device__ __forceinline__ void ld(const float* p, float& a, float& b) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        a = v.x; b = v.y;
    }
    static __device__ __forceinline__ void st(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
};
template <> struct Vec2<__half> {
    static __device__ __forceinline__ void ld(const __half* p, float& a, float& b) {
        const float2 v = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
        a = v.x; b = v.y;
    }
    static __device__ __forceinline__ void st(__half* p, float a, float b) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
};
template <> struct Vec2<__nv_bfloat16> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, float& a, float& b) {
        const float2 v = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
        a = v.x; b = v.y;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
};

// Pull for the node pair (x0, x0+1), x0 even: every population row is read as
// aligned pairs; the neighbour one column to the left (right) comes from the
// previous (next) lane's pair by warp shuffle, or from memory at a row or
// warp edge.  Every lane of the warp runs the shuffles (dead lanes re-read a
// valid pair), so the masks are always full.
template <int DIM, typename T>
__device__ __forceinline__ void pull2(const Params& p, const T* __restrict__ src, int x0, int y, int z, int n0,
                                      float* g0, float* g1) {
    using LT = Lat<DIM>;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int N = (int)p.n;
    const int lane = threadIdx.x & 31;
    const int ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
    const int zm = DIM == 3 ? wrap(z - 1, nz) : 0, zp = DIM == 3 ? wrap(z + 1, nz) : 0;
    const bool wall_lo = p.walls && (y == 1);
    const bool wall_hi = p.walls && (y == ny - 2);
    const bool left_edge = (lane == 0) || (x0 == 0);
    const bool right_edge = (lane == 31) || (x0 + 2 >= nx);
    const int xl = wrap(x0 - 1, nx), xr = x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2;
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const int cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
        const int ys = cy == 0 ? y : (cy > 0 ? ym : yp);
        const int zs = cz == 0 ? z : (cz > 0 ? zm : zp);
        const T* row = src + (size_t)i * N + ((size_t)zs * ny + ys) * nx;
        float a, b;
        Vec2<T>::ld(row + x0, a, b);
        if (cx == 1) {  // source x - 1: (x0 - 1, x0)
            float prev = __shfl_up_sync(0xffffffffu, b, 1);
            if (left_edge) prev = ldg_<T>(row + xl);
            b = a;
            a = prev;
        } else if (cx == -1) {  // source x + 1: (x0 + 1, x0 + 2)
            float next = __shfl_down_sync(0xffffffffu, a, 1);
            if (right_edge) next = ldg_<T>(row + xr);
            a = b;
            b = next;
        }
        const bool bb = (cy == 1 && wall_lo) || (cy == -1 && wall_hi);
        if (bb) Vec2<T>::ld(src + (size_t)LT::opp(i) * N + n0, a, b);
        g0[i] = a;
        g1[i] = b;
    }
}

template <int DIM, typename T, int SUB, bool CORR>
__device__ __forceinline__ void collide2_kernel_body(const VB& vb, const Params& p, const T* __restrict__ src,
                                                     T* __restrict__ dst, const float* __restrict__ vn,
                                                     const float* __restrict__ kolmo, DevState* st, VPtrs vk,
                                                     const float* __restrict__ betaf,
                                                     const float* __restrict__ mprow) {
    using LT = Lat<DIM>;
    const long long npair = p.n / 2;
    long long pi = (long long)vb.x * blockDim.x + threadIdx.x;
    const bool live = pi < npair;
    if (!live) pi = npair - 1;
    const int N = (int)p.n;
    const int n0 = (int)(2 * pi);
    const int x0 = n0 % p.nx;
    const int t = n0 / p.nx;
    const int y = t % p.ny;
    const int z = t / p.ny;
    float g0[LT::Q], g1[LT::Q];
    pull2<DIM, T>(p, src, x0, y, z, n0, g0, g1);
    if (!live) return;
    if (p.walls && (y == 0 || y == p.ny - 1)) return;
    float dx0 = 0.f, dy0 = 0.f, dz0 = 0.f, dx1 = 0.f, dy1 = 0.f, dz1 = 0.f;
    if (CORR) {
        sgs_increment<DIM>(p, vk, betaf, mprow, (size_t)n0, y, dx0, dy0, dz0);
        sgs_increment<DIM>(p, vk, betaf, mprow, (size_t)n0 + 1, y, dx1, dy1, dz1);
    }
    collide_node<DIM, SUB, (sizeof(T) == 4), CORR>(p, g0, x0, y, z, vn, kolmo, st, dx0, dy0, dz0);
    collide_node<DIM, SUB, (sizeof(T) == 4), CORR>(p, g1, x0 + 1, y, z, vn, kolmo, st, dx1, dy1, dz1);
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) Vec2<T>::st(dst + (size_t)i * N + n0, g0[i], g1[i]);
}
template <int DIM, typename T, int SUB, bool CORR>
struct collide2_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        collide2_kernel_body<DIM, T, SUB, CORR>(vb, b...);
    }
};
template <int DIM, typename T, int SUB, bool CORR>
__global__ void __launch_bounds__(128) collide2_kernel(Params p, const T* __restrict__ src, T* __restrict__ dst,
                                                       const float* __restrict__ vn, const float* __restrict__ kolmo,
                                                       DevState* st, VPtrs vk, const float* __restrict__ betaf,
                                                       const float* __restrict__ mprow) {
    collide2_kernel_body<DIM, T, SUB, CORR>(vb_hw(), p, src, dst, vn, kolmo, st, vk, betaf, mprow);
}

// f = f^eq(rho, u) on fluid nodes, 0 (= rest) on solid rows; inputs are the
// density deviation and the velocity as FP32 device arrays.
template <int DIM, typename T>
__global__ void init_feq_kernel(Params p, T* __restrict__ f, const float* __restrict__ drho_in,
                                const float* __restrict__ u) {
    using LT = Lat<DIM>;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n;
    const int y = (n / p.nx) % p.ny;
    const bool solid = p.walls && (y == 0 || y == p.ny - 1);
    const float dr = solid ? 0.f : drho_in[n];
    const float r = 1.0f + dr;
    const float ux = solid ? 0.f : u[n], uy = solid ? 0.f : u[(size_t)N + n];
    const float uz = (solid || DIM == 2) ? 0.f : u[(size_t)2 * N + n];
    const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const float cu = LT::cx(i) * ux + LT::cy(i) * uy + LT::cz(i) * uz;
        st_<T>(f + (size_t)i * N + n, solid ? 0.f : LT::w(i) * (dr + r * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu)));
    }
}

// density deviation and velocity sum c f / rho of a stored state
template <int DIM, typename T>
__global__ void macros_kernel(Params p, const T* __restrict__ f, float* __restrict__ drho, float* __restrict__ u) {
    using LT = Lat<DIM>;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.n) return;
    const int N = (int)p.n;
    const int y = (n / p.nx) % p.ny;
    if (p.walls && (y == 0 || y == p.ny - 1)) {
        drho[n] = 0.f;
        u[n] = 0.f; u[(size_t)N + n] = 0.f; u[(size_t)2 * N + n] = 0.f;
        return;
    }
    float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const float gi = ld_<T>(f + (size_t)i * N + n);
        dr += gi;
        jx += LT::cx(i) * gi;
        jy += LT::cy(i) * gi;
        jz += LT::cz(i) * gi;
    }
    const float inv = 1.0f / (1.0f + dr);
    drho[n] = dr;
    u[n] = jx * inv;
    u[(size_t)N + n] = jy * inv;
    u[(size_t)2 * N + n] = jz * inv;
}

// ---------------------------------------------------------------- launchers --
static inline unsigned grid_of(long long n, int b) { return (unsigned)((n + b - 1) / b); }

#define LBM_DISPATCH_STORAGE(p, FN, ...)                                                    \
    do {                                                                                    \
        if ((p).storage == LBM_STORAGE_FP16) FN<__half>(__VA_ARGS__);                       \
        else if ((p).storage == LBM_STORAGE_BF16) FN<__nv_bfloat16>(__VA_ARGS__);           \
        else FN<float>(__VA_ARGS__);                                                        \
    } while (0)

template <typename T>
static void do_init(const Params& p, const Layout& L, const float* drho, const float* u, int which, cudaStream_t s) {
    if (p.dim == 2)
        init_feq_kernel<2, T><<<grid_of(p.n, 256), 256, 0, s>>>(p, (T*)L.f[which], drho, u);
    else
        init_feq_kernel<3, T><<<grid_of(p.n, 256), 256, 0, s>>>(p, (T*)L.f[which], drho, u);
}
// predict_kernel for node pairs (nx even): the pair pull of collide2_kernel
// (aligned 2-element loads, x neighbours by warp shuffle), the same moments,
// 2-element stores.
template <int DIM, typename T, bool WV, bool WN>
__device__ __forceinline__ void predict2_kernel_body(const VB& vb, const Params& p, const T* __restrict__ src,
                                                     float* __restrict__ vps, float* __restrict__ vn,
                                                     const float* __restrict__ kolmo) {
    using LT = Lat<DIM>;
    const long long npair = p.n / 2;
    long long pi = (long long)vb.x * blockDim.x + threadIdx.x;
    const bool live = pi < npair;
    if (!live) pi = npair - 1;
    const size_t N = (size_t)p.n;
    const int n0 = (int)(2 * pi);
    const int x0 = n0 % p.nx;
    const int t = n0 / p.nx;
    const int y = t % p.ny;
    const int z = t / p.ny;
    float g0[LT::Q], g1[LT::Q];
    pull2<DIM, T>(p, src, x0, y, z, n0, g0, g1);
    if (!live) return;
    float2 vx = make_float2(0.f, 0.f), vy = vx, vz = vx, ux = vx, uy = vx, uz = vx;
    if (!(p.walls && (y == 0 || y == p.ny - 1))) {
        const Macro a = macros_of<DIM>(p, g0, kolmo, y);
        const Macro b = macros_of<DIM>(p, g1, kolmo, y);
        predictor_velocity(a, vx.x, vy.x, vz.x);
        predictor_velocity(b, vx.y, vy.y, vz.y);
        ux = make_float2(a.ux, b.ux);
        uy = make_float2(a.uy, b.uy);
        uz = make_float2(a.uz, b.uz);
    }
    if (WV) {
        *reinterpret_cast<float2*>(vps + n0) = vx;
        *reinterpret_cast<float2*>(vps + N + n0) = vy;
        if (DIM == 3) *reinterpret_cast<float2*>(vps + 2 * N + n0) = vz;
    }
    if (WN) {
        *reinterpret_cast<float2*>(vn + n0) = ux;
        *reinterpret_cast<float2*>(vn + N + n0) = uy;
        *reinterpret_cast<float2*>(vn + 2 * N + n0) = uz;
    }
}
template <int DIM, typename T, bool WV, bool WN>
struct predict2_kernel_op {
    static constexpr int NT = 128, MINB = 1;
    template <class... B>
    static __device__ __forceinline__ void run(const VB& vb, const B&... b) {
        predict2_kernel_body<DIM, T, WV, WN>(vb, b...);
    }
};
template <int DIM, typename T, bool WV, bool WN>
__global__ void __launch_bounds__(128) predict2_kernel(Params p, const T* __restrict__ src, float* __restrict__ vps,
                                                       float* __restrict__ vn, const float* __restrict__ kolmo) {
    predict2_kernel_body<DIM, T, WV, WN>(vb_hw(), p, src, vps, vn, kolmo);
}

cudaError_t launch_init_feq(const Params& p, const Layout& L, const float* drho, const float* u, int which,
                            cudaStream_t s) {
    LBM_DISPATCH_STORAGE(p, do_init, p, L, drho, u, which, s);
    return cudaGetLastError();
}

template <int DIM, typename T, bool WV, bool WN>
static void do_predict_d(const Params& p, const Layout& L, int src, cudaStream_t s) {
    const T* a = (const T*)L.f[src];
    if (p.nx % 2 == 0 && p.tune.predict_pair)  // node pairs (autotuned; single nodes read fewer bytes per load)
        go<predict2_kernel_op<DIM, T, WV, WN>>(predict2_kernel<DIM, T, WV, WN>, grid_of(p.n / 2, 128), 128, 0, s, p,
                                               a, L.vps, L.vn, L.kolmo);
    else
        go<predict_kernel_op<DIM, T, WV, WN>>(predict_kernel<DIM, T, WV, WN>, grid_of(p.n, 256), 256, 0, s, p, a,
                                              L.vps, L.vn, L.kolmo);
}
template <typename T>
static void do_predict(const Params& p, const Layout& L, int src, cudaStream_t s) {
    const bool wv = p.to_mode != LBM_TO_OFF, wn = p.substrate == LBM_SUBSTRATE_WALE;
    if (p.dim == 2) {
        if (wv && wn) do_predict_d<2, T, true, true>(p, L, src, s);
        else if (wv) do_predict_d<2, T, true, false>(p, L, src, s);
        else if (wn) do_predict_d<2, T, false, true>(p, L, src, s);
    } else {
        if (wv && wn) do_predict_d<3, T, true, true>(p, L, src, s);
        else if (wv) do_predict_d<3, T, true, false>(p, L, src, s);
        else if (wn) do_predict_d<3, T, false, true>(p, L, src, s);
    }
}
cudaError_t launch_predict(const Params& p, const Layout& L, int src, cudaStream_t s) {
    LBM_DISPATCH_STORAGE(p, do_predict, p, L, src, s);
    return cudaGetLastError();
}

bool corrector_runs(const Params& p) {
    return p.to_mode != LBM_TO_OFF && p.to_mode != LBM_TO_OBSERVE;
}

template <int DIM, typename T, int SUB, bool CORR>
static void do_collide_k(const Params& p, const Layout& L, int src, cudaStream_t s) {
    const T* a = (const T*)L.f[src];
    T* b = (T*)L.f[1 - src];
    VPtrs vk;
    for (int k = 0; k < kMaxQoi; ++k) vk.v[k] = nullptr;
    for (int k = 0; k < p.n_s; ++k) {
        const int slot = p.qoi_filter_slot[k];
        vk.v[k] = p.qoi_kind[k] == LBM_QOI_ENERGY ? L.rr[slot] : L.vz[slot];
    }
    if (p.nx % 2 == 0 && p.tune.collide_pair)  // node pairs: nx even keeps every pair inside one row, 2-aligned
        go<collide2_kernel_op<DIM, T, SUB, CORR>>(collide2_kernel<DIM, T, SUB, CORR>, grid_of(p.n / 2, 128), 128, 0, s,
                                                  p, a, b, L.vn, L.kolmo, L.st, vk, L.betaf, L.mprow);
    else if constexpr (collide_minb<DIM, T>() == 4)
        go<collide_kernel_op<DIM, T, SUB, CORR>>(collide4_kernel<DIM, T, SUB, CORR>, grid_of(p.n, 256), 256, 0, s, p,
                                                 a, b, L.vn, L.kolmo, L.st, vk, L.betaf, L.mprow);
    else
        go<collide_kernel_op<DIM, T, SUB, CORR>>(collide_kernel<DIM, T, SUB, CORR>, grid_of(p.n, 256), 256, 0, s, p,
                                                 a, b, L.vn, L.kolmo, L.st, vk, L.betaf, L.mprow);
}
template <int DIM, typename T, int SUB>
static void do_collide_s(const Params& p, const Layout& L, int src, cudaStream_t s) {
    if (corrector_runs(p)) do_collide_k<DIM, T, SUB, true>(p, L, src, s);
    else do_collide_k<DIM, T, SUB, false>(p, L, src, s);
}
template <int DIM, typename T>
static void do_collide_d(const Params& p, const Layout& L, int src, cudaStream_t s) {
    if (p.substrate == LBM_SUBSTRATE_SMAG) do_collide_s<DIM, T, LBM_SUBSTRATE_SMAG>(p, L, src, s);
    else if (p.substrate == LBM_SUBSTRATE_WALE) do_collide_s<DIM, T, LBM_SUBSTRATE_WALE>(p, L, src, s);
    else do_collide_s<DIM, T, LBM_SUBSTRATE_NONE>(p, L, src, s);
}
template <typename T>
static void do_collide(const Params& p, const Layout& L, int src, cudaStream_t s) {
    if (p.dim == 2) do_collide_d<2, T>(p, L, src, s);
    else do_collide_d<3, T>(p, L, src, s);
}
cudaError_t launch_collide(const Params& p, const Layout& L, int src, cudaStream_t s) {
    LBM_DISPATCH_STORAGE(p, do_collide, p, L, src, s);
    return cudaGetLastError();
}

template <typename T>
static void do_macros(const Params& p, const Layout& L, int which, float* drho, float* u, cudaStream_t s) {
    if (p.dim == 2)
        macros_kernel<2, T><<<grid_of(p.n, 256), 256, 0, s>>>(p, (const T*)L.f[which], drho, u);
    else
        macros_kernel<3, T><<<grid_of(p.n, 256), 256, 0, s>>>(p, (const T*)L.f[which], drho, u);
}
cudaError_t launch_macros(const Params& p, const Layout& L, int which, float* drho, float* u, cudaStream_t s) {
    LBM_DISPATCH_STORAGE(p, do_macros, p, L, which, drho, u, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------ projection --
// phi_m (Sec. 3, coarse graining) of the stored state onto an m-times coarser
// lattice: the density deviation and velocity sum c f / rho (as
// macros_kernel) at the HF nodes the projection reads, combined on the LF
// grid.  One thread per LF node; only the sampled HF nodes' populations are
// read (1/m^3 of the field in 3-D, 16/m^2 of it in 2-D for m >= 4).
template <int DIM, typename T>
__device__ __forceinline__ void node_macros(const T* __restrict__ f, size_t N, size_t n, float& dr, float& ux,
                                            float& uy, float& uz) {
    using LT = Lat<DIM>;
    float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const float gi = ldg_<T>(f + (size_t)i * N + n);
        r += gi;
        jx += LT::cx(i) * gi;
        jy += LT::cy(i) * gi;
        jz += LT::cz(i) * gi;
    }
    const float inv = 1.0f / (1.0f + r);
    dr = r;
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
}

// Keys' cubic convolution weight (a = -1/2) at distance t
__device__ __forceinline__ float keys_w(float t) {
    t = fabsf(t);
    if (t <= 1.f) return (1.5f * t - 2.5f) * t * t + 1.f;
    if (t < 2.f) return ((-0.5f * t + 2.5f) * t - 4.f) * t + 2.f;
    return 0.f;
}

// 2-D doubly periodic: bicubic interpolation at the LF block centres
// (m i + (m-1)/2, m j + (m-1)/2) in HF node units, over the 4 x 4 nearest
// HF nodes (taps of zero weight, all but one for odd m, are skipped)
template <typename T>
__global__ void __launch_bounds__(256) project2d_kernel(Params p, const T* __restrict__ f, int m, int nxl, int nyl,
                                                        float* __restrict__ drho, float* __restrict__ u) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = nxl * nyl;
    if (t >= nl) return;
    const int i = t % nxl, j = t / nxl;
    const size_t N = (size_t)p.n;
    const int half = (m - 1) / 2;
    const float frac = (m % 2 == 0) ? 0.5f : 0.f;  // X - floor(X)
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = keys_w(frac - (float)(k - 1));
    const int bx = m * i + half, by = m * j + half;
    float sr = 0.f, sx = 0.f, sy = 0.f;
    for (int b = 0; b < 4; ++b) {
        if (w[b] == 0.f) continue;
        const int ys = (by + b - 1 + p.ny) % p.ny;
        float rr = 0.f, rx = 0.f, ry = 0.f;
        for (int a = 0; a < 4; ++a) {
            if (w[a] == 0.f) continue;
            const int xs = (bx + a - 1 + p.nx) % p.nx;
            float dr, ux, uy, uz;
            node_macros<2, T>(f, N, (size_t)ys * p.nx + xs, dr, ux, uy, uz);
            rr = fmaf(w[a], dr, rr);
            rx = fmaf(w[a], ux, rx);
            ry = fmaf(w[a], uy, ry);
        }
        sr = fmaf(w[b], rr, sr);
        sx = fmaf(w[b], rx, sx);
        sy = fmaf(w[b], ry, sy);
    }
    drho[t] = sr;
    u[t] = sx;
    u[(size_t)nl + t] = sy;
    u[(size_t)2 * nl + t] = 0.f;
}

// 3-D channel: wall-anchored stride-m subsampling (odd m): LF fluid row j on
// HF row m j - (m-1)/2, solid rows on solid rows, x and z on the block centres
template <typename T>
__global__ void __launch_bounds__(256) project3d_kernel(Params p, const T* __restrict__ f, int m, int nxl, int nyl,
                                                        int nzl, float* __restrict__ drho, float* __restrict__ u) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nl = (long long)nxl * nyl * nzl;
    if (t >= nl) return;
    const int i = (int)(t % nxl);
    const long long r = t / nxl;
    const int j = (int)(r % nyl), k = (int)(r / nyl);
    float dr = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
    if (j > 0 && j < nyl - 1) {
        const int c = (m - 1) / 2;
        const size_t n = ((size_t)(m * k + c) * p.ny + (m * j - c)) * p.nx + (m * i + c);
        node_macros<3, T>(f, (size_t)p.n, n, dr, ux, uy, uz);
    }
    drho[t] = dr;
    u[t] = ux;
    u[nl + t] = uy;
    u[2 * nl + t] = uz;
}

template <typename T>
static void do_project(const Params& p, const Layout& L, int which, int m, int nxl, int nyl, int nzl, float* drho,
                       float* u, cudaStream_t s) {
    const long long nl = (long long)nxl * nyl * nzl;
    const unsigned grid = (unsigned)((nl + 255) / 256);
    if (p.dim == 2)
        project2d_kernel<T><<<grid, 256, 0, s>>>(p, (const T*)L.f[which], m, nxl, nyl, drho, u);
    else
        project3d_kernel<T><<<grid, 256, 0, s>>>(p, (const T*)L.f[which], m, nxl, nyl, nzl, drho, u);
}
cudaError_t launch_project(const Params& p, const Layout& L, int which, int m, int nxl, int nyl, int nzl,
                           float* drho, float* u, cudaStream_t s) {
    LBM_DISPATCH_STORAGE(p, do_project, p, L, which, m, nxl, nyl, nzl, drho, u, s);
    return cudaGetLastError();
}

}  // namespace lbm
