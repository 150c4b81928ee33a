// misa_alloy.cuh -- EAM passes for alloys (several atom types).
//
// With atom types the density of atom i sums the density function of each
// neighbour's type, the embedding function is that of i's type, and each
// pair has the pair function of its two types (Eq. eam_base); the force of
// pair (i, j) is [F'_i rho_{t_j}'(r) + F'_j rho_{t_i}'(r) + phi_{t_i t_j}'(r)]
// along r_hat (Eq. eam_force_ij).  Species are held per atom id, so atom
// moves between the site array and the run-away list need no bookkeeping.
//
// This file holds the alloy passes of the FP64 path (one thread per site)
// and, for both precisions, those of the run-away atoms (one warp per
// run-away): neighbours through the offset index and the run-away list
// (run-aways only from tiles flagged as within reach of one), spline tables
// read from global memory through L1, sums compensated in FP32 (plain in
// FP64) as in the single-type passes.  The FP32 path's array atoms go
// through the packed tile gathers of misa_alloy_packed.cuh.
#pragma once

#include "misa_adjoint.cuh"

namespace misa {

constexpr int kMaxSpecies = 4;

template <typename T>
struct AlloyArgs {
    const RepDesc *reps;  // replica table (density tile map's counts)
    int nrep;
    const int *sid;
    const T *ux, *uy, *uz;
    T *fp, *rho_out;
    double *e_out;
    T *ax, *ay, *az;
    double *vx, *vy, *vz;
    const int *ra_home, *ra_id;
    const T *ra_ux, *ra_uy, *ra_uz;
    T *ra_fp, *ra_rho;
    double *ra_e;
    T *ra_ax, *ra_ay, *ra_az;
    double *ra_vx, *ra_vy, *ra_vz;
    DevScalars *sc;
    const int8_t *atype;  // species per atom id
    int nsp, n;           // species; knots per table
    // coefficient tables, n entries per table: value (a, b, c, d) and
    // derivative (3a/h, 2b/h, c/h, 0) of each density function, value of each
    // embedding function, value and derivative of each pair function
    const Vec4<T> *tfv, *tfd, *tFv, *tpv, *tpd;
    T S, rc2, rfloor2, Srho, rho_max;
    double acc_conv;
    int kick, energy, nvec;
    const int *tile_flag;
    int tx, ty, tz;
    const int *ra_toff, *ra_tcnt, *ra_tlist;  // per-tile run-away index of the density map
    SplitN2 split[kMaxN2 + 1];
};

__device__ __forceinline__ int alloy_pair(int a, int b, int nsp)
{
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo * nsp - lo * (lo - 1) / 2 + (hi - lo);
}

template <typename T>
__device__ __forceinline__ int type_of(const AlloyArgs<T> &a, const AdjPair<T> &P)
{
    return a.atype[P.ra ? a.ra_id[P.j] : a.sid[P.j]];
}

template <typename T>
__device__ __forceinline__ T cubic_at(const Vec4<T> &c, T t)
{
    return ((c.x * t + c.y) * t + c.z) * t + c.w;
}

template <typename T>
__device__ __forceinline__ T quad_at(const Vec4<T> &c, T t)
{
    return (c.x * t + c.y) * t + c.z;
}

// rho_i = sum_j rho_{t_j}(r_ij)  (Sec. 2.2 step 1)
template <typename T>
struct AlloyRhoFn {
    const AlloyArgs<T> &a;
    Acc<T> rho;
    __device__ __forceinline__ void operator()(const AdjPair<T> &P)
    {
        rho.add(cubic_at<T>(a.tfv[(size_t)type_of(a, P) * a.n + P.seg], P.t));
    }
};

// force, half pair energy of atom i of type ti
template <typename T>
struct AlloyForceFn {
    const AlloyArgs<T> &a;
    int ti;
    T Fpi;
    Acc<T> fx, fy, fz;
    double ephi;
    __device__ __forceinline__ void operator()(const AdjPair<T> &P)
    {
        const int tj = type_of(a, P);
        const T Fpj = P.ra ? a.ra_fp[P.j] : a.fp[P.j];
        const size_t sg = (size_t)P.seg;
        const int pr = alloy_pair(ti, tj, a.nsp);
        const T dfi = quad_at<T>(a.tfd[(size_t)ti * a.n + sg], P.t);
        // the same function when the species agree: no second read or evaluation
        const T dfj = tj == ti ? dfi : quad_at<T>(a.tfd[(size_t)tj * a.n + sg], P.t);
        const T dph = quad_at<T>(a.tpd[(size_t)pr * a.n + sg], P.t);
        // Eq. eam_force_ij; the unit vector is zero below r_floor
        const T s = Fpi * dfj + Fpj * dfi + dph;
        fx.add(s * P.ex);
        fy.add(s * P.ey);
        fz.add(s * P.ez);
        if (a.energy) ephi += 0.5 * (double)cubic_at<T>(a.tpv[(size_t)pr * a.n + sg], P.t);
    }
};

template <typename T>
__device__ __forceinline__ T alloy_embed(const AlloyArgs<T> &a, int ti, T rho, T &dF, unsigned &st)
{
    return embed<T>(a.tFv + (size_t)ti * a.n, a.n - 1, a.Srho, a.rho_max, rho, dF, st);
}

// density pass for array atoms; grid.y = replica
template <typename T>
__global__ void k_alloy_density(AlloyArgs<T> a)
{
    const int r = blockIdx.y;
    const RepDesc rd = a.reps[r];
    const int nra = a.sc[r].n_ra;
    unsigned st = 0;
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        const int id = a.sid[s];
        if (id < 0) {
            a.fp[s] = 0;
            continue;
        }
        AlloyRhoFn<T> fn{a, Acc<T>()};
        visit_site<T>(a, rd, nra, ls, fn);
        const T rho = fn.rho.value();
        T dF;
        const T Fv = alloy_embed<T>(a, a.atype[id], rho, dF, st);
        a.fp[s] = dF;
        if (a.energy) {
            a.rho_out[s] = rho;
            a.e_out[s] = (double)Fv;
        }
    }
    if (st) atomicOr(&a.sc[0].status, st);
}

// density pass for run-aways; grid.y = replica
template <typename T>
__global__ void k_alloy_ra_density(AlloyArgs<T> a)
{
    const int r = blockIdx.y;
    const RepDesc rd = a.reps[r];
    const int nra = a.sc[r].n_ra;
    unsigned st = 0;
    MISA_RA_WARP_LOOP(nra, j) {
        const int g = rd.ra_base + j;
        AlloyRhoFn<T> fn{a, Acc<T>()};
        visit_ra<T>(a, rd, nra, j, fn);
        const T rho = (T)warp_sum((double)fn.rho.value());
        if ((threadIdx.x & 31) == 0) {
            T dF;
            const T Fv = alloy_embed<T>(a, a.atype[a.ra_id[g]], rho, dF, st);
            a.ra_fp[g] = dF;
            a.ra_rho[g] = rho;
            if (a.energy) a.ra_e[g] = (double)Fv;
        }
    }
    if (st) atomicOr(&a.sc[0].status, st);
}

// acceleration, closing half kick and the replica's max |v|
template <typename T>
__device__ __forceinline__ void alloy_finish(const AlloyArgs<T> &a, double hdt, const AlloyForceFn<T> &fn, T *ax, T *ay,
                                             T *az, double *vx, double *vy, double *vz, long long i,
                                             unsigned long long &vmax2, unsigned &st)
{
    const T gx = (T)((double)fn.fx.value() * a.acc_conv), gy = (T)((double)fn.fy.value() * a.acc_conv),
            gz = (T)((double)fn.fz.value() * a.acc_conv);
    ax[i] = gx;
    ay[i] = gy;
    az[i] = gz;
    if (!isfinite(gx) || !isfinite(gy) || !isfinite(gz)) st |= kStNonfinite;
    if (a.kick) {
        const double wx = fma(hdt, (double)gx, vx[i]), wy = fma(hdt, (double)gy, vy[i]), wz = fma(hdt, (double)gz, vz[i]);
        vx[i] = wx;
        vy[i] = wy;
        vz[i] = wz;
        const unsigned long long b = (unsigned long long)__double_as_longlong(wx * wx + wy * wy + wz * wz);
        vmax2 = b > vmax2 ? b : vmax2;
    }
}

// force pass for array atoms (Eq. eam_force_ij) + closing half kick; grid.y = replica
template <typename T>
__global__ void __launch_bounds__(256) k_alloy_force(AlloyArgs<T> a)
{
    __shared__ float red[kRedFloats];
    const int r = blockIdx.y;
    const RepDesc rd = a.reps[r];
    const int nra = a.sc[r].n_ra;
    const double hdt = 0.5 * a.sc[r].dt;
    unsigned st = 0;
    unsigned long long vmax2 = 0;
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        const int id = a.sid[s];
        if (id < 0) continue;
        AlloyForceFn<T> fn{a, a.atype[id], a.fp[s], Acc<T>(), Acc<T>(), Acc<T>(), 0.0};
        visit_site<T>(a, rd, nra, ls, fn);
        alloy_finish<T>(a, hdt, fn, a.ax, a.ay, a.az, a.vx, a.vy, a.vz, s, vmax2, st);
        if (a.energy) a.e_out[s] += fn.ephi;
    }
    if (a.kick) flush_vmax<256>(__longlong_as_double((long long)vmax2), red, a.sc + r);
    if (st) atomicOr(&a.sc[0].status, st);
}

// force pass for run-aways + closing half kick; grid.y = replica
template <typename T>
__global__ void __launch_bounds__(256) k_alloy_ra_force(AlloyArgs<T> a)
{
    __shared__ float red[kRedFloats];
    const int r = blockIdx.y;
    const RepDesc rd = a.reps[r];
    const int nra = a.sc[r].n_ra;
    const double hdt = 0.5 * a.sc[r].dt;
    unsigned st = 0;
    unsigned long long vmax2 = 0;
    MISA_RA_WARP_LOOP(nra, j) {
        const int g = rd.ra_base + j;
        AlloyForceFn<T> fn{a, a.atype[a.ra_id[g]], a.ra_fp[g], Acc<T>(), Acc<T>(), Acc<T>(), 0.0};
        visit_ra<T>(a, rd, nra, j, fn);
        fn.fx = Acc<T>{(T)warp_sum((double)fn.fx.value()), (T)0};
        fn.fy = Acc<T>{(T)warp_sum((double)fn.fy.value()), (T)0};
        fn.fz = Acc<T>{(T)warp_sum((double)fn.fz.value()), (T)0};
        fn.ephi = warp_sum(fn.ephi);
        if ((threadIdx.x & 31) == 0) {
            alloy_finish<T>(a, hdt, fn, a.ra_ax, a.ra_ay, a.ra_az, a.ra_vx, a.ra_vy, a.ra_vz, g, vmax2, st);
            if (a.energy) a.ra_e[g] += fn.ephi;
        }
    }
    if (a.kick) flush_vmax<256>(__longlong_as_double((long long)vmax2), red, a.sc + r);
    if (st) atomicOr(&a.sc[0].status, st);
}

// Coefficient tables of every alloy function (the local cubic Hermite of
// Sec. 4.1 as in k_spline_tables): nf density and embedding tables, np pair
// tables, n knots each.  One thread per (table, segment).
template <typename T>
__global__ void k_alloy_tables(const double *f, const double *F, const double *phi, int nsp, int npair, int n,
                               double hr, double hrho, Vec4<T> *tfv, Vec4<T> *tfd, Vec4<T> *tFv, Vec4<T> *tpv,
                               Vec4<T> *tpd)
{
    const long long total = (long long)(2 * nsp + npair) * n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int tab = (int)(q / n), k = (int)(q % n);
        const double *y;
        double h;
        Vec4<T> *val, *der;
        size_t o;
        if (tab < nsp) {
            y = f + (size_t)tab * n; h = hr; val = tfv; der = tfd; o = (size_t)tab * n;
        } else if (tab < 2 * nsp) {
            y = F + (size_t)(tab - nsp) * n; h = hrho; val = tFv; der = nullptr; o = (size_t)(tab - nsp) * n;
        } else {
            y = phi + (size_t)(tab - 2 * nsp) * n; h = hr; val = tpv; der = tpd; o = (size_t)(tab - 2 * nsp) * n;
        }
        if (k == n - 1) {
            val[o + k] = Vec4<T>{0, 0, 0, 0};
            if (der) der[o + k] = Vec4<T>{0, 0, 0, 0};
            continue;
        }
        const double m0 = knot_slope(y, n, h, k) * h, m1 = knot_slope(y, n, h, k + 1) * h;
        const double y0 = y[k], y1 = y[k + 1];
        const double ca = 2.0 * (y0 - y1) + m0 + m1, cb = 3.0 * (y1 - y0) - 2.0 * m0 - m1;
        val[o + k] = Vec4<T>{(T)ca, (T)cb, (T)m0, (T)y0};
        if (der) der[o + k] = Vec4<T>{(T)(3.0 * ca / h), (T)(2.0 * cb / h), (T)(m0 / h), (T)0};
    }
}

}  // namespace misa
