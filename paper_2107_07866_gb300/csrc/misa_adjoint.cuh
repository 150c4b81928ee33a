// misa_adjoint.cuh -- gradient of a force-matching + energy loss with respect
// to the knot values of the three spline tables (no counterpart in the
// paper; used to fit potentials).
//
// Per replica r with N_r atoms, forces F_i, energy E_r and targets:
//   L_r = (1/(3 N_r)) sum_i |F_i - Fref_i|^2 + ((E_r - Eref_r)/N_r)^2.
// With lambda_i = 2 (F_i - Fref_i)/(3 N_r), sum_i lambda_i . F_i is minus
// the derivative of E along the displacement field lambda, so the knot
// gradient of the force term is minus that directional derivative of
// dE/d(knot); the energy term adds c_e dE/d(knot), c_e = 2 (E_r - Eref_r)/N_r^2.
// The spline is linear in its knots (S(x) = sum_k w_k(x) y_k), so
//   phi knots: sum over ordered pairs of  c_e w_k/2 - dw_k D/2
//   f knots:   sum over ordered pairs of  c_e F'_i w_k - (F''_i Dl_i w_k + F'_i dw_k D)
//   F knots:   sum over atoms of          c_e w_k(rho_i) - dw_k(rho_i) Dl_i
// where D = d r_ij / d eps along lambda and Dl_i = sum_j f'(r_ij) D.
// Kernels: lambda (+ force-loss sums), Dl gather, gradient scatter into
// per-CTA bins in shared memory (in the handle's precision; FP32 bins in two
// copies, one per half warp, since shared FP32 atomics that collide within a
// warp are slow; their rounding, ~1e-6 of a bin, is far below the FP32
// gradient's own error).  A pair adds its Hermite weights to the value and
// slope bins of its segment's two end knots; one ordered FP64 reduction over
// CTAs, then the slope bins reach the knots through the slopes' difference
// stencils.  Pair arithmetic in the precision T of the handle.
#pragma once

#include "misa_md.cuh"
#include "misa_packed.cuh"

namespace misa {

// The upper half of every shell of kLVec: within a shell the vectors are
// sorted by (z, y, x), an order that negation reverses, so the second half
// holds exactly the vectors whose (z, y, x) is lexicographically positive.
// Walking it from every array site meets each unordered pair of array sites
// once.  Its prefix of n / 2 vectors covers the shells of kLVec's prefix of n.
constexpr LVecTable make_lvec_half()
{
    LVecTable t{};
    int c = 0;
    t.nshell = kLVec.nshell;
    for (int sh = 0; sh < kLVec.nshell; ++sh) {
        const int b = kLVec.shell_begin[sh], e = kLVec.shell_begin[sh + 1];
        t.shell_n2[sh] = kLVec.shell_n2[sh];
        t.shell_begin[sh] = c;
        for (int k = b + (e - b) / 2; k < e; ++k) t.v[c++] = kLVec.v[k];
    }
    t.shell_begin[t.nshell] = c;
    return t;
}

constexpr bool lvec_half_ok()
{
    for (int sh = 0; sh < kLVec.nshell; ++sh) {
        if ((kLVec.shell_begin[sh + 1] - kLVec.shell_begin[sh]) % 2) return false;
        for (int k = kLVec.shell_begin[sh]; k < kLVec.shell_begin[sh + 1]; ++k) {
            const LVec &o = kLVec.v[k];
            const bool pos = o.z > 0 || (o.z == 0 && (o.y > 0 || (o.y == 0 && o.x > 0)));
            const bool upper = k >= kLVec.shell_begin[sh] + (kLVec.shell_begin[sh + 1] - kLVec.shell_begin[sh]) / 2;
            if (pos != upper) return false;
        }
    }
    return true;
}

constexpr LVecTable kLVecHalf = make_lvec_half();
static_assert(lvec_half_ok() && kLVecHalf.shell_begin[kLVecHalf.nshell] == kNVec / 2,
              "each shell splits into a negative and a positive half");

// One offset of the per-site walks with what every candidate derives from
// it: the cell shifts along y and z from a site of parity 0 and 1, |n|^2,
// and n and |n|^2 as (exact) floating-point values, so that the walk
// computes no shift and converts no integer per candidate
struct WalkVec {
    int x, n2;
    int sy[2], sz[2];
    float fx, fy, fz, fn2;
};
struct WalkTable {
    WalkVec v[kNVec];
};

constexpr WalkTable make_walk(const LVecTable &t, int count)
{
    WalkTable w{};
    for (int k = 0; k < count; ++k) {
        const LVec &o = t.v[k];
        w.v[k] = WalkVec{o.x, o.n2, {cell_shift(0, o.y), cell_shift(1, o.y)}, {cell_shift(0, o.z), cell_shift(1, o.z)},
                         (float)o.x, (float)o.y, (float)o.z, (float)o.n2};
    }
    return w;
}
// the bcc lattice vectors (all, and the upper half of every shell) for the
// runtime-indexed walks
static __constant__ WalkTable c_walk = make_walk(kLVec, kNVec);
static __constant__ WalkTable c_walk_half = make_walk(kLVecHalf, kNVec / 2);

// |n| S = xint + xfrac for every |n|^2 <= kMaxN2 (S: knot index per lattice
// unit), split on the host in FP64 so that the FP32 pair geometry needs no
// FP64 arithmetic
struct SplitN2 {
    float nrm, xfrac;
    int xint, pad;
};

template <typename T>
struct AdjArgs {
    const RepDesc *reps;
    int nrep;
    const int *sid;
    const T *ux, *uy, *uz;
    const T *fp, *rho;
    const T *ax, *ay, *az;
    const int *ra_home, *ra_id;
    const T *ra_ux, *ra_uy, *ra_uz;
    const T *ra_fp, *ra_rho;
    const T *ra_ax, *ra_ay, *ra_az;
    const DevScalars *sc;
    const Vec4<T> *tab_d0, *tab_F;  // f' coefficients (x, y, z of d0), F value coefficients
    int n;                          // knots per table
    T S;                            // knot index per lattice unit of r
    T hr, hrho, rho_max, rc2, rfloor2, half;
    T inv_hr, inv_hrho;  // 1/hr, 1/hrho
    double acc_conv, inv_acc_conv;
    const double *Fref;   // 3 per atom id
    const double *Eref;   // per replica
    const double *Etot;   // per replica
    T *lam_x, *lam_y, *lam_z;        // per site (pooled)
    T *ra_lx, *ra_ly, *ra_lz;        // per run-away slot
    T *dl, *ra_dl;                   // D_lambda rho per site / run-away slot
    T *cw;  // per site: ce F'_i - F''_i D_lambda rho_i, the weight of the knot values in the f scatter
    int nvec;                        // offsets within rc + 2 skin (prefix of kLVec)
    const int *tile_flag;            // null: every site scans the run-away list
    int tx, ty, tz;
    const int *ra_toff, *ra_tcnt, *ra_tlist;  // per-tile run-away index of that map (or null)
    SplitN2 split[kMaxN2 + 1];
};

// one pair seen from atom i: |r| in lattice units, unit vector i -> j, the
// spline segment and t of r, and where atom j lives (array site or run-away
// slot, pooled indices)
template <typename T>
struct AdjPair {
    T r, ex, ey, ez;
    bool ra;
    long long j;
    int seg;
    T t;
    bool floor_hit;
};

// Pair geometry from the integer lattice vector n between the two sites and
// d = u_j - u_i.  The spline argument x = r S is formed as |n| S (FP64,
// split into integer and fraction) plus (r - |n|) S with
// r - |n| = q / (r + |n|), q = (2n + d).d: full precision in t also in FP32
// (x is near 2000, where a plain FP32 r S keeps only ~1e-4 of t).
// (n given as exact floating-point values nxf, nyf, nzf and |n|^2 as n2
// and n2f, so that a walk over a fixed offset table converts nothing)
template <typename T, typename A>
__device__ __forceinline__ bool adj_pair_n(const A &a, T nxf, T nyf, T nzf, int n2, T n2f, T dx, T dy, T dz, bool ra,
                                           long long j, AdjPair<T> &P)
{
    const T q = ((T)2 * nxf + dx) * dx + ((T)2 * nyf + dy) * dy + ((T)2 * nzf + dz) * dz;
    const T r2 = n2f + q;
    if (!(r2 < a.rc2)) return false;
    const T rx = nxf + dx, ry = nyf + dy, rz = nzf + dz;
    P.ra = ra;
    P.j = j;
    P.floor_hit = r2 < a.rfloor2;
    T r, inv;
    if constexpr (sizeof(T) == 4) {  // approximate reciprocal square root, as in the tile gathers
        const T rr2 = P.floor_hit ? a.rfloor2 : r2;
        const T rs = rsqrt_approx(rr2);
        r = rr2 * rs;
        inv = P.floor_hit ? (T)0 : rs;
    } else {  // FP32 seed and Newton steps (rsqrt_nr): no FP64 square root or division
        const T rr2 = P.floor_hit ? a.rfloor2 : r2;
        const T rs = rsqrt_nr(rr2);
        r = rr2 * rs;
        inv = P.floor_hit ? (T)0 : rs;
    }
    P.r = r;
    P.ex = rx * inv;
    P.ey = ry * inv;
    P.ez = rz * inv;
    if (P.floor_hit || n2 == 0) {
        const double x = (double)r * (double)a.S;
        const double fl = floor(x);
        P.seg = (int)fl;
        P.t = (T)(x - fl);
    } else if constexpr (sizeof(T) == 4) {
        const SplitN2 sp = a.split[n2];
        const T dr = q * rcp_approx(r + (T)sp.nrm);
        const T x = (T)sp.xfrac + dr * a.S;
        const T fl = floor(x);
        P.seg = sp.xint + (int)fl;
        P.t = x - fl;
    } else {  // FP64: r S carries the full precision t needs
        const T x = r * a.S;
        const T fl = floor(x);
        P.seg = (int)fl;
        P.t = x - fl;
    }
    if (P.seg < 0) {
        P.seg = 0;
        P.t = 0;
    }
    if (P.seg > a.n - 2) {
        P.seg = a.n - 2;
        P.t = 1;
    }
    return true;
}

template <typename T, typename A>
__device__ __forceinline__ bool adj_pair(const A &a, int nx, int ny, int nz, T dx, T dy, T dz, bool ra, long long j,
                                         AdjPair<T> &P)
{
    const int n2 = nx * nx + ny * ny + nz * nz;
    return adj_pair_n<T>(a, (T)nx, (T)ny, (T)nz, n2, (T)n2, dx, dy, dz, ra, j, P);
}

// Visits the array-site neighbours j of array atom i (replica-local site
// ls, displacement ui, half-lattice x index x2 and cell row cy, cz) inside
// rc through the offset vectors: all of them, or with HALF only those along
// the positive half of each shell (every unordered pair of array sites once
// over all i).
template <typename T, bool HALF, typename A, typename Fn>
__device__ __forceinline__ void visit_site_array(const A &a, const RepDesc &rd, T uix, T uiy, T uiz, int x2, int cy,
                                                 int cz, Fn &fn)
{
    const int p = x2 & 1;
    const int nv = HALF ? a.nvec / 2 : a.nvec;
#pragma unroll 4
    for (int k = 0; k < nv; ++k) {
        const WalkVec &o = HALF ? c_walk_half.v[k] : c_walk.v[k];
        const int tx = wrap_near(x2 + o.x, 2 * rd.nx);
        const int ty = wrap_near(cy + o.sy[p], rd.ny);
        const int tz = wrap_near(cz + o.sz[p], rd.nz);
        // 32-bit index arithmetic: a handle holds fewer than 2^31 sites
        const int t = (int)rd.site_base + ((tz * rd.ny + ty) * rd.nx) * 2 + tx;
        if (a.sid[t] < 0) continue;
        AdjPair<T> P;
        if (adj_pair_n<T>(a, (T)o.fx, (T)o.fy, (T)o.fz, o.n2, (T)o.fn2, a.ux[t] - uix, a.uy[t] - uiy, a.uz[t] - uiz,
                          false, t, P))
            fn(P);
    }
}

// Visits the run-aways j within rc of array atom i: those of the site's
// tile index entry (list order) when the list is longer than kRaScanMax,
// else the whole list (only from tiles flagged as within reach of a
// run-away when a.tile_flag is set; rd's tile counts are those tiles').
template <typename T, typename A, typename Fn>
__device__ __forceinline__ void visit_site_ra(const A &a, const RepDesc &rd, int nra, long long ls, T uix, T uiy,
                                              T uiz, int x2, int cy, int cz, Fn &fn)
{
    if (nra == 0) return;
    const int *jl = nullptr;
    int nj = nra;
    if (a.tile_flag) {
        const int tl = rd.tile_base + ((cz / a.tz) * rd.nty + cy / a.ty) * rd.ntx + (x2 >> 1) / a.tx;
        const int f = a.tile_flag[tl];
        if (!f) return;
        if (f == 1 && a.ra_tlist && nra > kRaScanMax) {
            jl = a.ra_tlist + a.ra_toff[tl];
            nj = a.ra_tcnt[tl];
        }
    }
    int X, Y, Z;
    site_lat32((int)ls, rd.nx, rd.ny, X, Y, Z);
    const int Lx = 2 * rd.nx, Ly = 2 * rd.ny, Lz = 2 * rd.nz;
    for (int jq = 0; jq < nj; ++jq) {
        const int j = jl ? jl[jq] : jq;
        const int g = rd.ra_base + j;
        int Xj, Yj, Zj;
        site_lat32(a.ra_home[g], rd.nx, rd.ny, Xj, Yj, Zj);
        int nx_ = Xj - X, ny_ = Yj - Y, nz_ = Zj - Z;
        nx_ -= (nx_ > rd.nx) ? Lx : 0;
        nx_ += (nx_ < -rd.nx) ? Lx : 0;
        ny_ -= (ny_ > rd.ny) ? Ly : 0;
        ny_ += (ny_ < -rd.ny) ? Ly : 0;
        nz_ -= (nz_ > rd.nz) ? Lz : 0;
        nz_ += (nz_ < -rd.nz) ? Lz : 0;
        AdjPair<T> P;
        if (adj_pair<T>(a, nx_, ny_, nz_, a.ra_ux[g] - uix, a.ra_uy[g] - uiy, a.ra_uz[g] - uiz, true, g, P)) fn(P);
    }
}

// where array site ls sits: its displacement and lattice row
template <typename T, typename A>
__device__ __forceinline__ void site_here(const A &a, const RepDesc &rd, long long ls, T &uix, T &uiy, T &uiz,
                                          int &x2, int &cy, int &cz)
{
    const long long s = rd.site_base + ls;
    uix = a.ux[s]; uiy = a.uy[s]; uiz = a.uz[s];
    const int li = (int)ls;  // fewer than 2^31 sites: 32-bit division
    x2 = li % (2 * rd.nx);
    const int q = li / (2 * rd.nx);
    cy = q % rd.ny;
    cz = q / rd.ny;
}

// Visits every neighbour j of array atom i (replica-local site ls) inside
// rc: array atoms through the offset vectors, then the run-aways.
template <typename T, typename A, typename Fn>
__device__ __forceinline__ void visit_site(const A &a, const RepDesc &rd, int nra, long long ls, Fn &fn)
{
    T uix, uiy, uiz;
    int x2, cy, cz;
    site_here<T>(a, rd, ls, uix, uiy, uiz, x2, cy, cz);
    visit_site_array<T, false>(a, rd, uix, uiy, uiz, x2, cy, cz, fn);
    visit_site_ra<T>(a, rd, nra, ls, uix, uiy, uiz, x2, cy, cz, fn);
}

// One warp per run-away: j runs over the warps of the grid (warp-uniform).
#define MISA_RA_WARP_LOOP(nra, j)                                                                       \
    for (int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < (nra);                        \
         j += (int)((gridDim.x * blockDim.x) >> 5))

// Visits the neighbours of run-away j (pooled slot g): array sites in a
// 7-cell window around its home site, then the other run-aways.  The
// candidates are dealt out over the 32 lanes of a warp (lane takes every
// 32nd); the caller sums the lanes' partial results with warp_sum (FP64).
template <typename T, typename A, typename Fn>
__device__ __forceinline__ void visit_ra(const A &a, const RepDesc &rd, int nra, int jl, Fn &fn)
{
    const int lane = threadIdx.x & 31;
    const int g = rd.ra_base + jl;
    int X, Y, Z;
    site_lat32(a.ra_home[g], rd.nx, rd.ny, X, Y, Z);
    const int hp = X & 1;
    const int hcx = X >> 1, hcy = (Y - hp) >> 1, hcz = (Z - hp) >> 1;
    const T ujx = a.ra_ux[g], ujy = a.ra_uy[g], ujz = a.ra_uz[g];
    const int wx = rd.nx < 7 ? rd.nx : 7, wy = rd.ny < 7 ? rd.ny : 7, wz = rd.nz < 7 ? rd.nz : 7;
    for (int c = lane; c < wx * wy * wz * 2; c += 32) {
        const int qq = c & 1, rr = c >> 1;
        const int ox = rr % wx, oy = (rr / wx) % wy, oz = rr / (wx * wy);
        const int cx = hcx - 3 + ox, cy = hcy - 3 + oy, cz = hcz - 3 + oz;
        const int t = (int)rd.site_base + ((wrap_near(cz, rd.nz) * rd.ny + wrap_near(cy, rd.ny)) * rd.nx + wrap_near(cx, rd.nx)) * 2 + qq;
        if (a.sid[t] < 0) continue;
        AdjPair<T> P;
        if (adj_pair<T>(a, 2 * cx + qq - X, 2 * cy + qq - Y, 2 * cz + qq - Z, a.ux[t] - ujx, a.uy[t] - ujy,
                        a.uz[t] - ujz, false, t, P))
            fn(P);
    }
    const int Lx = 2 * rd.nx, Ly = 2 * rd.ny, Lz = 2 * rd.nz;
    // the other run-aways: the home tile's index entry (lane l takes the list
    // indices k = l mod 32, ascending) when the list is longer than
    // kRaScanMax, else the whole list
    const int *kl = nullptr;
    if (a.tile_flag && a.ra_tlist && nra > kRaScanMax) {
        const int tl = rd.tile_base + ((hcz / a.tz) * rd.nty + hcy / a.ty) * rd.ntx + hcx / a.tx;
        if (a.tile_flag[tl] == 1) kl = a.ra_tlist + a.ra_toff[tl];
        if (kl) nra = a.ra_tcnt[tl];
    }
    for (int kq = kl ? 0 : lane; kq < nra; kq += kl ? 1 : 32) {
        const int k = kl ? kl[kq] : kq;
        if (kl && (k & 31) != lane) continue;
        if (k == jl) continue;
        const int gk = rd.ra_base + k;
        int Xk, Yk, Zk;
        site_lat32(a.ra_home[gk], rd.nx, rd.ny, Xk, Yk, Zk);
        int nx_ = Xk - X, ny_ = Yk - Y, nz_ = Zk - Z;
        nx_ -= (nx_ > rd.nx) ? Lx : 0;
        nx_ += (nx_ < -rd.nx) ? Lx : 0;
        ny_ -= (ny_ > rd.ny) ? Ly : 0;
        ny_ += (ny_ < -rd.ny) ? Ly : 0;
        nz_ -= (nz_ > rd.nz) ? Lz : 0;
        nz_ += (nz_ < -rd.nz) ? Lz : 0;
        AdjPair<T> P;
        if (adj_pair<T>(a, nx_, ny_, nz_, a.ra_ux[gk] - ujx, a.ra_uy[gk] - ujy, a.ra_uz[gk] - ujz, true, gk, P)) fn(P);
    }
}

// Weights of knots s-2 .. s+3 in S(x) and dS/dx at x = (s + t) h for the
// local Hermite spline (slopes: 4th-order central differences inside,
// 2nd order at the two outer knots of each end).
template <typename T>
__device__ __forceinline__ void basis6(int s, T t, int n, T inv_h, T w[6], T dw[6])
{
    const T t2 = t * t, t3 = t2 * t;
    const T c0 = 2 * t3 - 3 * t2 + 1, c1 = t3 - 2 * t2 + t, c2 = -2 * t3 + 3 * t2, c3 = t3 - t2;
    const T d0 = (6 * t2 - 6 * t) * inv_h, d1 = (3 * t2 - 4 * t + 1) * inv_h, d2 = (-6 * t2 + 6 * t) * inv_h,
            d3 = (3 * t2 - 2 * t) * inv_h;
    if (s >= 2 && s <= n - 4) {
        // both knot slopes from the 4th-order stencil (y_{k-2} - 8 y_{k-1} +
        // 8 y_{k+1} - y_{k+2}) / 12: the weights of knots s-2 .. s+3 in closed form
        const T a = (T)(1.0 / 12.0), b = (T)(8.0 / 12.0);
        w[0] = c1 * a;
        w[1] = c3 * a - c1 * b;
        w[2] = c0 - c3 * b;
        w[3] = c2 + c1 * b;
        w[4] = c3 * b - c1 * a;
        w[5] = -(c3 * a);
        dw[0] = d1 * a;
        dw[1] = d3 * a - d1 * b;
        dw[2] = d0 - d3 * b;
        dw[3] = d2 + d1 * b;
        dw[4] = d3 * b - d1 * a;
        dw[5] = -(d3 * a);
        return;
    }
    for (int q = 0; q < 6; ++q) {
        w[q] = 0;
        dw[q] = 0;
    }
    w[2] += c0;
    dw[2] += d0;
    w[3] += c2;
    dw[3] += d2;
    // h * slope of knot k = sum_l st_l y_l (h cancels against the 1/h of the stencil)
    for (int e = 0; e < 2; ++e) {
        const int k = s + e;
        const T cm = e == 0 ? c1 : c3, dm = e == 0 ? d1 : d3;
        int ks[4];
        T st[4];
        int ns;
        if (k == 0) {
            ks[0] = 0; st[0] = (T)-1.5; ks[1] = 1; st[1] = (T)2; ks[2] = 2; st[2] = (T)-0.5; ns = 3;
        } else if (k == n - 1) {
            ks[0] = n - 1; st[0] = (T)1.5; ks[1] = n - 2; st[1] = (T)-2; ks[2] = n - 3; st[2] = (T)0.5; ns = 3;
        } else if (k == 1 || k == n - 2) {
            ks[0] = k + 1; st[0] = (T)0.5; ks[1] = k - 1; st[1] = (T)-0.5; ns = 2;
        } else {
            ks[0] = k - 2; st[0] = (T)(1.0 / 12.0); ks[1] = k - 1; st[1] = (T)(-8.0 / 12.0);
            ks[2] = k + 1; st[2] = (T)(8.0 / 12.0); ks[3] = k + 2; st[3] = (T)(-1.0 / 12.0); ns = 4;
        }
        for (int q = 0; q < ns; ++q) {
            const int j = ks[q] - (s - 2);
            w[j] += cm * st[q];
            dw[j] += dm * st[q];
        }
    }
}

// spline segment and t of x on a grid of spacing h (n knots)
template <typename T>
__device__ __forceinline__ int seg_t(T x, T inv_h, int n, T &t)
{
    const T u = x * inv_h;
    int s = (int)floor(u);
    s = s < 0 ? 0 : (s > n - 2 ? n - 2 : s);
    t = u - (T)s;
    return s;
}

// lambda_i = 2 (F_i - Fref_i)/(3 N_r) per site and run-away; per-(replica,
// block) partial sums of |F_i - Fref_i|^2.  grid.y = replica.
template <typename T>
__global__ void k_adj_lambda(AdjArgs<T> a, double *partial)
{
    const int r = blockIdx.y;
    const RepDesc rd = a.reps[r];
    const double c = 2.0 / (3.0 * (double)rd.ns);
    double acc = 0.0;
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        const int id = a.sid[s];
        if (id < 0) continue;
        const double fx = (double)a.ax[s] * a.inv_acc_conv - a.Fref[3LL * id];
        const double fy = (double)a.ay[s] * a.inv_acc_conv - a.Fref[3LL * id + 1];
        const double fz = (double)a.az[s] * a.inv_acc_conv - a.Fref[3LL * id + 2];
        acc += fx * fx + fy * fy + fz * fz;
        a.lam_x[s] = (T)(c * fx);
        a.lam_y[s] = (T)(c * fy);
        a.lam_z[s] = (T)(c * fz);
    }
    const int nra = a.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        const int id = a.ra_id[g];
        const double fx = (double)a.ra_ax[g] * a.inv_acc_conv - a.Fref[3LL * id];
        const double fy = (double)a.ra_ay[g] * a.inv_acc_conv - a.Fref[3LL * id + 1];
        const double fz = (double)a.ra_az[g] * a.inv_acc_conv - a.Fref[3LL * id + 2];
        acc += fx * fx + fy * fy + fz * fz;
        a.ra_lx[g] = (T)(c * fx);
        a.ra_ly[g] = (T)(c * fy);
        a.ra_lz[g] = (T)(c * fz);
    }
    __shared__ double sw[32];
    acc = warp_sum<double>(acc);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
        partial[(size_t)r * gridDim.x + blockIdx.x] = t;
    }
}

template <typename T>
struct LamOf {
    const AdjArgs<T> &a;
    __device__ __forceinline__ void get(const AdjPair<T> &P, T &lx, T &ly, T &lz) const
    {
        if (P.ra) {
            lx = a.ra_lx[P.j]; ly = a.ra_ly[P.j]; lz = a.ra_lz[P.j];
        } else {
            lx = a.lam_x[P.j]; ly = a.lam_y[P.j]; lz = a.lam_z[P.j];
        }
    }
};

// D_lambda r_ij = rhat_ij . (lambda_i - lambda_j) = e . (lambda_j - lambda_i)
// with e the unit vector from i to j
template <typename T>
struct DlFn {
    const AdjArgs<T> &a;
    T lix, liy, liz;
    Acc<T> acc;
    __device__ __forceinline__ void operator()(const AdjPair<T> &P)
    {
        if (P.floor_hit) return;  // direction undefined: no derivative
        T ljx, ljy, ljz;
        LamOf<T>{a}.get(P, ljx, ljy, ljz);
        const T t = P.t;
        const Vec4<T> c = a.tab_d0[P.seg];
        const T dfr = (c.x * t + c.y) * t + c.z;
        const T D = P.ex * (ljx - lix) + P.ey * (ljy - liy) + P.ez * (ljz - liz);
        acc.add(dfr * D);
    }
};

template <typename T>
__device__ __forceinline__ T energy_weight(const AdjArgs<T> &a, int r, const RepDesc &rd)
{
    const double Nr = (double)rd.ns;
    return (T)(2.0 * (a.Etot[r] - a.Eref[r]) / (Nr * Nr));
}

template <typename T>
__device__ __forceinline__ T embed_dd(const AdjArgs<T> &a, T rho);

// three 256-thread CTAs per SM for FP32 (79 registers, no spills): the walk
// is bound by load latency and gains from the extra warps
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_adj_dl(AdjArgs<T> a)
{
    const int r = blockIdx.y;
    const RepDesc rd = a.reps[r];
    const int nra = a.sc[r].n_ra;
    const T ce = energy_weight<T>(a, r, rd);
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        if (a.sid[s] < 0) continue;
        DlFn<T> fn{a, a.lam_x[s], a.lam_y[s], a.lam_z[s], Acc<T>()};
        visit_site<T>(a, rd, nra, ls, fn);
        const T dl = fn.acc.value();
        a.dl[s] = dl;
        a.cw[s] = ce * a.fp[s] - embed_dd<T>(a, a.rho[s]) * dl;
    }
    MISA_RA_WARP_LOOP(nra, j) {
        const int g = rd.ra_base + j;
        DlFn<T> fn{a, a.ra_lx[g], a.ra_ly[g], a.ra_lz[g], Acc<T>()};
        visit_ra<T>(a, rd, nra, j, fn);
        const double dl = warp_sum((double)fn.acc.value());
        if ((threadIdx.x & 31) == 0) a.ra_dl[g] = (T)dl;
    }
}

// per-pair scatter into the CTA's bins: bins[0, n) f knots, [n, 2n) phi
// knots, [2n, 3n) F knots
template <typename T>
struct GradFn {
    const AdjArgs<T> &a;
    T *bins;
    T lix, liy, liz;
    T cw;   // ce F'_i - F''_i D_lrho_i: weight of the knot values in the f scatter
    T Fpi;  // F'_i: weight of the knot-derivative term
    T hce;  // ce / 2
    __device__ __forceinline__ void operator()(const AdjPair<T> &P)
    {
        T ljx, ljy, ljz;
        LamOf<T>{a}.get(P, ljx, ljy, ljz);
        // unit vector is zero below r_floor: no derivative term there
        const T D = P.ex * (ljx - lix) + P.ey * (ljy - liy) + P.ez * (ljz - liz);
        const T fD = Fpi * D, hD = (T)0.5 * D;
        // Hermite weights of the segment ends' values (c0, c2) and h-scaled
        // slopes (c1, c3), and their r derivatives; the slopes' knot stencils
        // are applied once, after the sum over CTAs (k_adj_stencil)
        const T t = P.t, t2 = t * t, t3 = t2 * t, ih = a.inv_hr;
        const T c0 = 2 * t3 - 3 * t2 + 1, c1 = t3 - 2 * t2 + t, c2 = -2 * t3 + 3 * t2, c3 = t3 - t2;
        const T d0 = (6 * t2 - 6 * t) * ih, d1 = (3 * t2 - 4 * t + 1) * ih, d2 = (-6 * t2 + 6 * t) * ih,
                d3 = (3 * t2 - 2 * t) * ih;
        const int sg = P.seg;  // 0 <= sg <= n - 2
        T *Yf = bins, *Yp = bins + a.n, *Mf = bins + 3 * a.n, *Mp = bins + 4 * a.n;
        atomicAdd(&Yf[sg], cw * c0 - fD * d0);
        atomicAdd(&Yf[sg + 1], cw * c2 - fD * d2);
        atomicAdd(&Mf[sg], cw * c1 - fD * d1);
        atomicAdd(&Mf[sg + 1], cw * c3 - fD * d3);
        atomicAdd(&Yp[sg], hce * c0 - hD * d0);
        atomicAdd(&Yp[sg + 1], hce * c2 - hD * d2);
        atomicAdd(&Mp[sg], hce * c1 - hD * d1);
        atomicAdd(&Mp[sg + 1], hce * c3 - hD * d3);
    }
};

// The same scatter for an unordered pair of array sites, visited once (the
// half walk): both directions share r, its segment and t, and D (e and
// lambda_j - lambda_i both change sign), so their terms add up to one
// scatter with the weights summed: cw_i + cw_j and (F'_i + F'_j) D for f,
// ce and D for phi.
template <typename T>
struct GradPairFn {
    const AdjArgs<T> &a;
    T *bins;
    T lix, liy, liz;
    T cwi, Fpi, ce;
    __device__ __forceinline__ void operator()(const AdjPair<T> &P)
    {
        const T ljx = a.lam_x[P.j], ljy = a.lam_y[P.j], ljz = a.lam_z[P.j];
        const T cw = cwi + a.cw[P.j];
        const T D = P.ex * (ljx - lix) + P.ey * (ljy - liy) + P.ez * (ljz - liz);
        const T fD = (Fpi + a.fp[P.j]) * D;
        const T t = P.t, t2 = t * t, t3 = t2 * t, ih = a.inv_hr;
        const T c0 = 2 * t3 - 3 * t2 + 1, c1 = t3 - 2 * t2 + t, c2 = -2 * t3 + 3 * t2, c3 = t3 - t2;
        const T d0 = (6 * t2 - 6 * t) * ih, d1 = (3 * t2 - 4 * t + 1) * ih, d2 = (-6 * t2 + 6 * t) * ih,
                d3 = (3 * t2 - 2 * t) * ih;
        const int sg = P.seg;
        T *Yf = bins, *Yp = bins + a.n, *Mf = bins + 3 * a.n, *Mp = bins + 4 * a.n;
        atomicAdd(&Yf[sg], cw * c0 - fD * d0);
        atomicAdd(&Yf[sg + 1], cw * c2 - fD * d2);
        atomicAdd(&Mf[sg], cw * c1 - fD * d1);
        atomicAdd(&Mf[sg + 1], cw * c3 - fD * d3);
        atomicAdd(&Yp[sg], ce * c0 - D * d0);
        atomicAdd(&Yp[sg + 1], ce * c2 - D * d2);
        atomicAdd(&Mp[sg], ce * c1 - D * d1);
        atomicAdd(&Mp[sg + 1], ce * c3 - D * d3);
    }
};

// F'' of the embedding spline at rho (0 on the linear tail)
template <typename T>
__device__ __forceinline__ T embed_dd(const AdjArgs<T> &a, T rho)
{
    if (rho > a.rho_max) return 0;
    if (rho < 0) rho = 0;
    T t;
    const int sg = seg_t<T>(rho, a.inv_hrho, a.n, t);
    const Vec4<T> c = a.tab_F[sg];
    return (6 * c.x * t + 2 * c.y) * (a.inv_hrho * a.inv_hrho);
}

template <typename T>
__device__ __forceinline__ void embed_bins(const AdjArgs<T> &a, T *bins, T rho, T ce, T dli)
{
    T w[6], dw[6];
    int sg;
    T ex = 0;
    if (rho > a.rho_max) {
        sg = a.n - 2;
        basis6<T>(sg, (T)1, a.n, a.inv_hrho, w, dw);
        ex = rho - a.rho_max;
    } else {
        T t;
        sg = seg_t<T>(rho < 0 ? (T)0 : rho, a.inv_hrho, a.n, t);
        basis6<T>(sg, t, a.n, a.inv_hrho, w, dw);
    }
    for (int q = 0; q < 6; ++q) {
        const int k = sg - 2 + q;
        if (k < 0 || k >= a.n) continue;
        const T g = ce * (w[q] + dw[q] * ex) - dw[q] * dli;
        if (g != (T)0) atomicAdd(&bins[2 * a.n + k], g);
    }
}

// gradient scatter: grid (blocks, replica); each CTA zeroes its 5n bins in
// shared memory ([0, n) f values, [n, 2n) phi values, [2n, 3n) F knots, [3n,
// 4n) f slopes, [4n, 5n) phi slopes), scatters its atoms' pair terms with
// shared-memory atomics, then writes the bins to partial[cta][5n] (FP64)
// copies = 2: the bins in two copies, one per half warp (shared-memory FP32
// atomics that collide within a warp are several times slower than distinct
// ones); 1 when two copies do not fit.
template <typename T>
constexpr int kGradThreads = sizeof(T) == 4 ? 1024 : 256;

template <typename T>
__global__ void __launch_bounds__(kGradThreads<T>) k_adj_grad(AdjArgs<T> a, double *partial, int copies)
{
    extern __shared__ __align__(16) unsigned char bin_smem[];
    const int r = blockIdx.y;
    const RepDesc rd = a.reps[r];
    const int nra = a.sc[r].n_ra;
    const int nb = 5 * a.n;
    for (int k = threadIdx.x; k < copies * nb; k += blockDim.x) reinterpret_cast<T *>(bin_smem)[k] = (T)0;
    T *bins = reinterpret_cast<T *>(bin_smem) + (copies == 2 && (threadIdx.x & 16) ? nb : 0);
    __syncthreads();
    const T ce = energy_weight<T>(a, r, rd);
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        if (a.sid[s] < 0) continue;
        const T Fpi = a.fp[s], cwi = a.cw[s];
        T uix, uiy, uiz;
        int x2, cy, cz;
        site_here<T>(a, rd, ls, uix, uiy, uiz, x2, cy, cz);
        // array-site pairs once (half walk, both directions' terms), the
        // site's run-away pairs from this side (the run-away's walk below
        // adds the other direction)
        GradPairFn<T> fp2{a, bins, a.lam_x[s], a.lam_y[s], a.lam_z[s], cwi, Fpi, ce};
        visit_site_array<T, true>(a, rd, uix, uiy, uiz, x2, cy, cz, fp2);
        GradFn<T> fn{a, bins, a.lam_x[s], a.lam_y[s], a.lam_z[s], cwi, Fpi, (T)0.5 * ce};
        visit_site_ra<T>(a, rd, nra, ls, uix, uiy, uiz, x2, cy, cz, fn);
        embed_bins<T>(a, bins, a.rho[s], ce, a.dl[s]);
    }
    MISA_RA_WARP_LOOP(nra, j) {
        const int g = rd.ra_base + j;
        const T rho = a.ra_rho[g];
        const T Fpi = a.ra_fp[g];
        GradFn<T> fn{a, bins, a.ra_lx[g], a.ra_ly[g], a.ra_lz[g], ce * Fpi - embed_dd<T>(a, rho) * a.ra_dl[g], Fpi,
                     (T)0.5 * ce};
        visit_ra<T>(a, rd, nra, j, fn);
        if ((threadIdx.x & 31) == 0) embed_bins<T>(a, bins, rho, ce, a.ra_dl[g]);
    }
    __syncthreads();
    double *out = partial + ((size_t)r * gridDim.x + blockIdx.x) * nb;
    const T *b0 = reinterpret_cast<const T *>(bin_smem);
    for (int k = threadIdx.x; k < nb; k += blockDim.x)
        out[k] = copies == 2 ? (double)b0[k] + (double)b0[nb + k] : (double)b0[k];
}

// grad[k] = sum over CTAs of partial[cta][k] in a fixed order: a block of
// 32 x 8 threads takes 32 knots; thread row y sums CTAs y, y + 8, ... in
// order, then the 8 row sums are added in row order.  Launch with blockDim
// (32, 8) and ceil(nb / 32) blocks.
static __global__ void __launch_bounds__(256) k_adj_reduce(const double *partial, int ncta, int nb, double *grad)
{
    __shared__ double rows[8][33];
    const int k = blockIdx.x * 32 + threadIdx.x;
    double s = 0.0;
    if (k < nb)
        for (int c = threadIdx.y; c < ncta; c += 8) s += partial[(size_t)c * nb + k];
    rows[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && k < nb) {
        double t = rows[0][threadIdx.x];
        for (int y = 1; y < 8; ++y) t += rows[y][threadIdx.x];
        grad[k] = t;
    }
}

// h * slope of knot k = sum_j slope_weight(k, j) y_j: the knot slopes of
// the spline (4th-order central differences inside, 2nd order at the two
// outer knots of each end)
__device__ __forceinline__ double slope_weight(int k, int j, int n)
{
    if (k == 0) return j == 0 ? -1.5 : j == 1 ? 2.0 : j == 2 ? -0.5 : 0.0;
    if (k == n - 1) return j == n - 1 ? 1.5 : j == n - 2 ? -2.0 : j == n - 3 ? 0.5 : 0.0;
    if (k == 1 || k == n - 2) return j == k + 1 ? 0.5 : j == k - 1 ? -0.5 : 0.0;
    const int d = j - k;
    return d == -2 ? 1.0 / 12.0 : d == -1 ? -8.0 / 12.0 : d == 1 ? 8.0 / 12.0 : d == 2 ? -1.0 / 12.0 : 0.0;
}

// Knot gradient from the summed bins (sum[5n], layout of k_adj_grad):
// d/dy_j of the f and phi tables = value bin j + sum over the slopes k
// within two knots of j of slope bin k * slope_weight(k, j); F knots as
// summed.
static __global__ void k_adj_stencil(const double *sum, int n, double *grad)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 3 * n; q += gridDim.x * blockDim.x) {
        double g = sum[q];
        if (q < 2 * n) {
            const int tab = q / n, j = q - tab * n;
            const double *M = sum + (size_t)(3 + tab) * n;
            for (int k = j - 2; k <= j + 2; ++k)
                if (k >= 0 && k < n) g += M[k] * slope_weight(k, j, n);
        }
        grad[q] = g;
    }
}

}  // namespace misa
