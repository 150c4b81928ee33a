// misa_md.cuh -- integration, lattice-list maintenance and read-out kernels.
//
// Velocity Verlet (Fig. 1, read as kick-drift-kick) with the adaptive
// timestep of the cascade feature list (Sec. 1), the hash update of Alg. 2
// (read with a skin: an array atom farther than skin from its site joins the
// run-away list at once; run-aways move back into empty nearest sites every
// reassign period, lowest atom id first), the run-away part of Alg. 1 (each
// run-away gathers over array sites around it and over the other
// run-aways), PKA insertion (Sec. 5.1), and per-atom read-out.
#pragma once

#include "misa_kernels.cuh"

namespace misa {

constexpr int kSortMax = 16384;  // run-away list capacity limit (single-CTA sort)

template <typename T>
struct MdArgs {
    int nx, ny, nz;
    long long ns;
    int *sid;                      // atom id per site, -1 vacant
    double *ux, *uy, *uz;          // displacement (lattice units); vacant: kVacant
    T *sx, *sy, *sz;               // precision-T shadow of u read by the gather (aliases u in FP64)
    double *vx, *vy, *vz;
    T *ax, *ay, *az;
    T *fp, *rho;
    double *esite;
    int *claim;
    // run-away list (capacity cap); tmp arrays are the permutation scratch
    int cap;
    int *ra_home, *ra_id;
    double *ra_ux, *ra_uy, *ra_uz;
    T *ra_sx, *ra_sy, *ra_sz;
    double *ra_vx, *ra_vy, *ra_vz;
    T *ra_ax, *ra_ay, *ra_az;
    T *ra_fp, *ra_rho;
    double *ra_e;
    int *t_home, *t_id;
    double *t_u[3], *t_v[3];
    T *t_s[3], *t_a[3];
    int *tile_flag;
    int tx, ty, tz, ntx, nty, ntz;
    DevScalars *sc;
    double half;      // a0/2 (A per lattice unit)
    double inv_half;
    double skin2;     // skin^2, lattice units
    double dt_max, dx_max;
    int reassign_period;
    double acc_conv;  // eV/A -> A/fs^2
    double mass;
};

// site id <-> lattice coordinates (lattice units: (2cx + p, 2cy + p, 2cz + p))
__device__ __forceinline__ void site_lat(long long s, int nx, int ny, int &X, int &Y, int &Z)
{
    int x2 = (int)(s % (2 * nx));
    long long r = s / (2 * nx);
    int cy = (int)(r % ny), cz = (int)(r / ny);
    int p = x2 & 1;
    X = x2;
    Y = 2 * cy + p;
    Z = 2 * cz + p;
}

__device__ __forceinline__ int wrapi(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// The hash function of Sec. 3 in lattice units: nearest site of the point
// P (unwrapped lattice coords).  Candidates: nearest corner (all coords even)
// and nearest centre (all odd); the closer wins, a tie goes to the lower id.
// Returns the site id and writes the displacement P - site (lattice units).
__device__ __forceinline__ long long nearest_site(double Px, double Py, double Pz, int nx, int ny, int nz, double &ux,
                                                  double &uy, double &uz)
{
    double cx = 2.0 * floor(Px * 0.5 + 0.5), cy = 2.0 * floor(Py * 0.5 + 0.5), cz = 2.0 * floor(Pz * 0.5 + 0.5);
    double ex = 2.0 * floor(Px * 0.5) + 1.0, ey = 2.0 * floor(Py * 0.5) + 1.0, ez = 2.0 * floor(Pz * 0.5) + 1.0;
    double dc = (Px - cx) * (Px - cx) + (Py - cy) * (Py - cy) + (Pz - cz) * (Pz - cz);
    double de = (Px - ex) * (Px - ex) + (Py - ey) * (Py - ey) + (Pz - ez) * (Pz - ez);
    auto sid_of = [&](double X, double Y, double Z) -> long long {
        int p = ((long long)X) & 1;
        int cxx = wrapi((int)floor(X * 0.5), nx), cyy = wrapi((int)floor(Y * 0.5), ny), czz = wrapi((int)floor(Z * 0.5), nz);
        return (((long long)czz * ny + cyy) * nx + cxx) * 2 + p;
    };
    long long idc = sid_of(cx, cy, cz), ide = sid_of(ex, ey, ez);
    bool corner = dc < de || (dc == de && idc < ide);
    if (corner) {
        ux = Px - cx; uy = Py - cy; uz = Pz - cz;
        return idc;
    }
    ux = Px - ex; uy = Py - ey; uz = Pz - ez;
    return ide;
}

// ---------------------------------------------------------------------------
// step bookkeeping
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_begin_step(MdArgs<T> m)
{
    DevScalars *sc = m.sc;
    double vmax = __longlong_as_double((long long)sc->vmax_bits);
    double dt = m.dt_max;
    if (m.dx_max > 0.0 && vmax > 0.0) dt = fmin(m.dt_max, m.dx_max / vmax);
    sc->dt = dt;
    sc->vacc_bits = 0ull;
    sc->n_ra_old = sc->n_ra;
    sc->n_new = 0;
    sc->dirty = 0;
}

// Empties the run-away list bookkeeping before an explicit state is loaded
// (step count and time are kept).
template <typename T>
__global__ void k_reset_list(MdArgs<T> m)
{
    DevScalars *sc = m.sc;
    sc->n_ra = 0;
    sc->n_ra_old = 0;
    sc->n_new = 0;
    sc->dirty = 1;
    sc->status = 0u;
    sc->vmax_bits = 0ull;
    sc->vacc_bits = 0ull;
}

template <typename T>
__global__ void k_end_step(MdArgs<T> m)
{
    DevScalars *sc = m.sc;
    sc->t += sc->dt;
    sc->step += 1;
    sc->vmax_bits = sc->vacc_bits;
}

// Opening half kick + drift of array atoms (FP64).  An atom leaving its
// skin is demoted to the run-away list (Alg. 2 part 1, skin reading).
template <typename T>
__global__ void k_kick_drift(MdArgs<T> m)
{
    DevScalars *sc = m.sc;
    const double dt = sc->dt, hdt = 0.5 * dt, dtl = dt * m.inv_half;
    const int base = sc->n_ra_old;
    const float skin2f = (float)m.skin2;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x) {
        int id = m.sid[s];
        if (id < 0) continue;
        // FP64 integration; the skin test (a storage decision) in FP32
        const double vx = fma(hdt, (double)m.ax[s], m.vx[s]);
        const double vy = fma(hdt, (double)m.ay[s], m.vy[s]);
        const double vz = fma(hdt, (double)m.az[s], m.vz[s]);
        const double ux = fma(dtl, vx, m.ux[s]);
        const double uy = fma(dtl, vy, m.uy[s]);
        const double uz = fma(dtl, vz, m.uz[s]);
        const float fx = (float)ux, fy = (float)uy, fz = (float)uz;
        bool out;
        if constexpr (sizeof(T) == 4) out = fx * fx + fy * fy + fz * fz > skin2f;
        else out = ux * ux + uy * uy + uz * uz > m.skin2;
        if (out) {
            int slot = atomicAdd(&sc->n_new, 1);
            int j = base + slot;
            if (j < m.cap) {
                int X, Y, Z;
                site_lat(s, m.nx, m.ny, X, Y, Z);
                double rx, ry, rz;
                long long h = nearest_site(X + ux, Y + uy, Z + uz, m.nx, m.ny, m.nz, rx, ry, rz);
                m.ra_home[j] = (int)h;
                m.ra_id[j] = id;
                m.ra_ux[j] = rx; m.ra_uy[j] = ry; m.ra_uz[j] = rz;
                m.ra_sx[j] = (T)rx; m.ra_sy[j] = (T)ry; m.ra_sz[j] = (T)rz;
                m.ra_vx[j] = vx; m.ra_vy[j] = vy; m.ra_vz[j] = vz;
                m.ra_ax[j] = m.ax[s]; m.ra_ay[j] = m.ay[s]; m.ra_az[j] = m.az[s];
                m.sid[s] = -1;
                m.ux[s] = kVacant; m.uy[s] = kVacant; m.uz[s] = kVacant;
                if ((void *)m.sx != (void *)m.ux) {
                    m.sx[s] = (T)kVacant; m.sy[s] = (T)kVacant; m.sz[s] = (T)kVacant;
                }
                continue;
            }
            atomicOr(&sc->status, kStRunawayOverflow);
        }
        m.vx[s] = vx; m.vy[s] = vy; m.vz[s] = vz;
        m.ux[s] = ux; m.uy[s] = uy; m.uz[s] = uz;
        if constexpr (sizeof(T) == 4) {
            m.sx[s] = fx; m.sy[s] = fy; m.sz[s] = fz;
        }
    }
}

// Opening half kick + drift of the run-aways present before this step;
// each is re-homed on its (new) nearest site.
template <typename T>
__global__ void k_ra_kick_drift(MdArgs<T> m)
{
    DevScalars *sc = m.sc;
    const double dt = sc->dt, hdt = 0.5 * dt;
    const int n = sc->n_ra_old;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double vx = m.ra_vx[j] + hdt * (double)m.ra_ax[j];
        double vy = m.ra_vy[j] + hdt * (double)m.ra_ay[j];
        double vz = m.ra_vz[j] + hdt * (double)m.ra_az[j];
        int X, Y, Z;
        site_lat(m.ra_home[j], m.nx, m.ny, X, Y, Z);
        double Px = X + m.ra_ux[j] + dt * vx * m.inv_half;
        double Py = Y + m.ra_uy[j] + dt * vy * m.inv_half;
        double Pz = Z + m.ra_uz[j] + dt * vz * m.inv_half;
        double rx, ry, rz;
        long long h = nearest_site(Px, Py, Pz, m.nx, m.ny, m.nz, rx, ry, rz);
        m.ra_home[j] = (int)h;
        m.ra_ux[j] = rx; m.ra_uy[j] = ry; m.ra_uz[j] = rz;
        m.ra_sx[j] = (T)rx; m.ra_sy[j] = (T)ry; m.ra_sz[j] = (T)rz;
        m.ra_vx[j] = vx; m.ra_vy[j] = vy; m.ra_vz[j] = vz;
    }
}

// Alg. 2 part 2: a run-away whose nearest site is empty and which lies
// within the skin of it claims the site; the lowest atom id wins.
template <typename T>
__global__ void k_reassign_claim(MdArgs<T> m, int force)
{
    DevScalars *sc = m.sc;
    if (!force && (sc->step + 1) % m.reassign_period != 0) return;
    int n = sc->n_ra_old + min(sc->n_new, m.cap - sc->n_ra_old);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int h = m.ra_home[j];
        double u2 = m.ra_ux[j] * m.ra_ux[j] + m.ra_uy[j] * m.ra_uy[j] + m.ra_uz[j] * m.ra_uz[j];
        if (m.sid[h] < 0 && u2 <= m.skin2) {
            atomicMin(&m.claim[h], m.ra_id[j]);
            sc->dirty = 1;
        }
    }
}

template <typename T>
__global__ void k_reassign_promote(MdArgs<T> m, int force)
{
    DevScalars *sc = m.sc;
    if (!force && (sc->step + 1) % m.reassign_period != 0) return;
    int n = sc->n_ra_old + min(sc->n_new, m.cap - sc->n_ra_old);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int h = m.ra_home[j];
        int id = m.ra_id[j];
        if (m.claim[h] == id && m.sid[h] < 0) {
            m.sid[h] = id;
            m.ux[h] = m.ra_ux[j]; m.uy[h] = m.ra_uy[j]; m.uz[h] = m.ra_uz[j];
            if ((void *)m.sx != (void *)m.ux) {
                m.sx[h] = (T)m.ra_ux[j]; m.sy[h] = (T)m.ra_uy[j]; m.sz[h] = (T)m.ra_uz[j];
            }
            m.vx[h] = m.ra_vx[j]; m.vy[h] = m.ra_vy[j]; m.vz[h] = m.ra_vz[j];
            m.ax[h] = m.ra_ax[j]; m.ay[h] = m.ra_ay[j]; m.az[h] = m.ra_az[j];
            m.ra_id[j] = -1;  // removed from the list by k_ra_sort
        }
    }
}

// Rebuilds the run-away list in ascending atom id (deterministic order for
// every gather that scans it), dropping promoted entries; resets the site
// claims.  One CTA, bitonic sort of (id, index) keys in shared memory.
template <typename T>
__global__ void __launch_bounds__(1024) k_ra_sort(MdArgs<T> m)
{
    extern __shared__ unsigned long long skey[];
    DevScalars *sc = m.sc;
    int nnew = sc->n_new;
    int n = sc->n_ra_old + min(nnew, m.cap - sc->n_ra_old);
    if (nnew == 0 && sc->dirty == 0) return;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned long long key = ~0ull;
        if (i < n) {
            int id = m.ra_id[i];
            key = ((unsigned long long)(id < 0 ? 0xFFFFFFFFu : (unsigned)id) << 32) | (unsigned)i;
            m.claim[m.ra_home[i]] = 0x7FFFFFFF;
        }
        skey[i] = key;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    unsigned long long a = skey[i], b = skey[l];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        skey[i] = b;
                        skey[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int local = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if ((skey[i] >> 32) != 0xFFFFFFFFull) ++local;
    atomicAdd(&s_cnt, local);
    __syncthreads();
    int cnt = s_cnt;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        int src = (int)(skey[i] & 0xFFFFFFFFu);
        m.t_home[i] = m.ra_home[src];
        m.t_id[i] = m.ra_id[src];
        m.t_u[0][i] = m.ra_ux[src]; m.t_u[1][i] = m.ra_uy[src]; m.t_u[2][i] = m.ra_uz[src];
        m.t_v[0][i] = m.ra_vx[src]; m.t_v[1][i] = m.ra_vy[src]; m.t_v[2][i] = m.ra_vz[src];
        m.t_s[0][i] = m.ra_sx[src]; m.t_s[1][i] = m.ra_sy[src]; m.t_s[2][i] = m.ra_sz[src];
        m.t_a[0][i] = m.ra_ax[src]; m.t_a[1][i] = m.ra_ay[src]; m.t_a[2][i] = m.ra_az[src];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        m.ra_home[i] = m.t_home[i];
        m.ra_id[i] = m.t_id[i];
        m.ra_ux[i] = m.t_u[0][i]; m.ra_uy[i] = m.t_u[1][i]; m.ra_uz[i] = m.t_u[2][i];
        m.ra_vx[i] = m.t_v[0][i]; m.ra_vy[i] = m.t_v[1][i]; m.ra_vz[i] = m.t_v[2][i];
        m.ra_sx[i] = m.t_s[0][i]; m.ra_sy[i] = m.t_s[1][i]; m.ra_sz[i] = m.t_s[2][i];
        m.ra_ax[i] = m.t_a[0][i]; m.ra_ay[i] = m.t_a[1][i]; m.ra_az[i] = m.t_a[2][i];
    }
    if (threadIdx.x == 0) {
        sc->n_ra = cnt;
        if (sc->n_ra_old + nnew > m.cap) atomicOr(&sc->status, kStRunawayOverflow);
    }
}

// Marks every tile within 3 cells of a run-away's home cell: those tiles'
// CTAs scan the run-away list.  tile_flag is zeroed before.
template <typename T>
__global__ void k_mark_tiles(MdArgs<T> m)
{
    int n = m.sc->n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int h = m.ra_home[j];
        int x2 = h % (2 * m.nx);
        int r = h / (2 * m.nx);
        int c[3] = {x2 >> 1, r % m.ny, r / m.ny};
        int nn[3] = {m.nx, m.ny, m.nz};
        int tt[3] = {m.tx, m.ty, m.tz};
        int tl[3][8], nt[3];
        for (int d = 0; d < 3; ++d) {
            nt[d] = 0;
            int w = nn[d] < 7 ? nn[d] : 7;
            for (int o = 0; o < w; ++o) {
                int cc = wrapi(c[d] - 3 + o, nn[d]);
                int t = cc / tt[d];
                bool seen = false;
                for (int q = 0; q < nt[d]; ++q) seen |= (tl[d][q] == t);
                if (!seen) tl[d][nt[d]++] = t;
            }
        }
        for (int a = 0; a < nt[2]; ++a)
            for (int b = 0; b < nt[1]; ++b)
                for (int e = 0; e < nt[0]; ++e) m.tile_flag[(tl[2][a] * m.nty + tl[1][b]) * m.ntx + tl[0][e]] = 1;
    }
}

// ---------------------------------------------------------------------------
// run-away gather (Alg. 1 parts 2-3): one warp per run-away atom
// ---------------------------------------------------------------------------

template <typename T>
struct RaGatherArgs {
    GatherArgs<T> g;  // tables, box, site arrays
    const int *sid;
    const T *ra_sx, *ra_sy, *ra_sz;
    T *ra_fp, *ra_rho;
    double *ra_e;
    T *ra_ax, *ra_ay, *ra_az;
    double *ra_vx, *ra_vy, *ra_vz;
    int energy;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// mode 0: density (+F, F'), mode 1: force (+kick)
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_ra_gather(const __grid_constant__ RaGatherArgs<T> ra)
{
    const GatherArgs<T> &a = ra.g;
    const int n = a.sc->n_ra;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const double hdt = 0.5 * a.sc->dt;
    unsigned st = 0;
    double vmax2 = 0.0;
    const int Lx = 2 * a.nx, Ly = 2 * a.ny, Lz = 2 * a.nz;
    for (int j = warp; j < n; j += nwarps) {
        int h = a.ra_home[j];
        int X, Y, Z;
        site_lat(h, a.nx, a.ny, X, Y, Z);
        const int hp = X & 1;
        const int hcx = X >> 1, hcy = (Y - hp) >> 1, hcz = (Z - hp) >> 1;
        T ujx = ra.ra_sx[j], ujy = ra.ra_sy[j], ujz = ra.ra_sz[j];
        T fpj = MODE == 1 ? ra.ra_fp[j] : (T)0;
        Acc<T> s0, s1, s2;
        double ephi = 0.0;
        const int wx = a.nx < 7 ? a.nx : 7, wy = a.ny < 7 ? a.ny : 7, wz = a.nz < 7 ? a.nz : 7;
        const int W = wx * wy * wz * 2;
        for (int c = lane; c < W; c += 32) {
            int q = c & 1;
            int r = c >> 1;
            int ox = r % wx, oy = (r / wx) % wy, oz = r / (wx * wy);
            int cx = hcx - 3 + ox, cy = hcy - 3 + oy, cz = hcz - 3 + oz;
            long long s = (((long long)wrapi(cz, a.nz) * a.ny + wrapi(cy, a.ny)) * a.nx + wrapi(cx, a.nx)) * 2 + q;
            if (ra.sid[s] < 0) continue;
            int nx_ = 2 * cx + q - X, ny_ = 2 * cy + q - Y, nz_ = 2 * cz + q - Z;
            T dx = a.ux[s] - ujx, dy = a.uy[s] - ujy, dz = a.uz[s] - ujz;
            T qq = (dx + (T)(2 * nx_)) * dx + (dy + (T)(2 * ny_)) * dy + (dz + (T)(2 * nz_)) * dz;
            T r2 = (T)(nx_ * nx_ + ny_ * ny_ + nz_ * nz_) + qq;
            if (r2 < a.rc2) {
                int seg;
                T t, rinv;
                bool fh;
                direct_arg<T>(r2, a.S, a.rfloor2, seg, t, rinv, fh);
                seg = clamp_seg<T>(seg, a.nseg, t);
                if (fh) st |= kStRfloor;
                if (MODE == 0) {
                    Vec4<T> cf = a.tab_f[seg];
                    s0.add(((cf.x * t + cf.y) * t + cf.z) * t + cf.w);
                } else {
                    Vec4<T> c0 = a.tab_d0[seg];
                    Vec2<T> c1 = a.tab_d1[seg];
                    T dfr = (c0.x * t + c0.y) * t + c0.z;
                    T dph = (c0.w * t + c1.x) * t + c1.y;
                    T coef = (fpj + a.fp[s]) * dfr + dph;
                    T sc = fh ? (T)0 : coef * rinv;
                    s0.add(sc * (dx + (T)nx_));
                    s1.add(sc * (dy + (T)ny_));
                    s2.add(sc * (dz + (T)nz_));
                    if (ra.energy) {
                        Vec4<T> cp = a.tab_phi[seg];
                        ephi += 0.5 * (double)(((cp.x * t + cp.y) * t + cp.z) * t + cp.w);
                    }
                }
            }
        }
        for (int k = lane; k < n; k += 32) {
            if (k == j) continue;
            int Xk, Yk, Zk;
            site_lat(a.ra_home[k], a.nx, a.ny, Xk, Yk, Zk);
            int nx_ = Xk - X, ny_ = Yk - Y, nz_ = Zk - Z;
            nx_ -= (nx_ > a.nx) ? Lx : 0;
            nx_ += (nx_ < -a.nx) ? Lx : 0;
            ny_ -= (ny_ > a.ny) ? Ly : 0;
            ny_ += (ny_ < -a.ny) ? Ly : 0;
            nz_ -= (nz_ > a.nz) ? Lz : 0;
            nz_ += (nz_ < -a.nz) ? Lz : 0;
            T dx = ra.ra_sx[k] - ujx, dy = ra.ra_sy[k] - ujy, dz = ra.ra_sz[k] - ujz;
            T qq = (dx + (T)(2 * nx_)) * dx + (dy + (T)(2 * ny_)) * dy + (dz + (T)(2 * nz_)) * dz;
            T r2 = (T)(nx_ * nx_ + ny_ * ny_ + nz_ * nz_) + qq;
            if (r2 < a.rc2) {
                int seg;
                T t, rinv;
                bool fh;
                direct_arg<T>(r2, a.S, a.rfloor2, seg, t, rinv, fh);
                seg = clamp_seg<T>(seg, a.nseg, t);
                if (fh) st |= kStRfloor;
                if (MODE == 0) {
                    Vec4<T> cf = a.tab_f[seg];
                    s0.add(((cf.x * t + cf.y) * t + cf.z) * t + cf.w);
                } else {
                    Vec4<T> c0 = a.tab_d0[seg];
                    Vec2<T> c1 = a.tab_d1[seg];
                    T dfr = (c0.x * t + c0.y) * t + c0.z;
                    T dph = (c0.w * t + c1.x) * t + c1.y;
                    T coef = (fpj + ra.ra_fp[k]) * dfr + dph;
                    T sc = fh ? (T)0 : coef * rinv;
                    s0.add(sc * (dx + (T)nx_));
                    s1.add(sc * (dy + (T)ny_));
                    s2.add(sc * (dz + (T)nz_));
                    if (ra.energy) {
                        Vec4<T> cp = a.tab_phi[seg];
                        ephi += 0.5 * (double)(((cp.x * t + cp.y) * t + cp.z) * t + cp.w);
                    }
                }
            }
        }
        if (MODE == 0) {
            T rh = warp_sum<T>(s0.value());
            if (lane == 0) {
                T dF;
                T Fv = embed<T>(a.tab_F, a.nseg, a.Srho, a.rho_max, rh, dF, st);
                ra.ra_fp[j] = dF;
                if (ra.energy) {
                    ra.ra_rho[j] = rh;
                    ra.ra_e[j] = (double)Fv;
                }
            }
        } else {
            T fx = warp_sum<T>(s0.value()), fy = warp_sum<T>(s1.value()), fz = warp_sum<T>(s2.value());
            double eph = warp_sum<double>(ephi);
            if (lane == 0) {
                double conv = a.acc_conv;
                double gx = (double)fx * conv, gy = (double)fy * conv, gz = (double)fz * conv;
                ra.ra_ax[j] = (T)gx;
                ra.ra_ay[j] = (T)gy;
                ra.ra_az[j] = (T)gz;
                if (!isfinite(gx) || !isfinite(gy) || !isfinite(gz)) st |= kStNonfinite;
                if (a.kick) {
                    double vx = ra.ra_vx[j] + hdt * (double)(T)gx;
                    double vy = ra.ra_vy[j] + hdt * (double)(T)gy;
                    double vz = ra.ra_vz[j] + hdt * (double)(T)gz;
                    ra.ra_vx[j] = vx;
                    ra.ra_vy[j] = vy;
                    ra.ra_vz[j] = vz;
                    double v2 = vx * vx + vy * vy + vz * vz;
                    vmax2 = v2 > vmax2 ? v2 : vmax2;
                }
                if (ra.energy) ra.ra_e[j] += eph;
            }
        }
    }
    if (st) atomicOr(&a.sc->status, st);
    if (MODE == 1 && a.kick && lane == 0 && vmax2 > 0.0)
        atomicMax(&a.sc->vacc_bits, (unsigned long long)__double_as_longlong(sqrt(vmax2)));
}

// ---------------------------------------------------------------------------
// state set-up and read-out
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_init_crystal(MdArgs<T> m)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x) {
        m.sid[s] = (int)s;
        m.ux[s] = 0.0; m.uy[s] = 0.0; m.uz[s] = 0.0;
        if ((void *)m.sx != (void *)m.ux) {
            m.sx[s] = (T)0; m.sy[s] = (T)0; m.sz[s] = (T)0;
        }
        m.vx[s] = 0.0; m.vy[s] = 0.0; m.vz[s] = 0.0;
        m.ax[s] = (T)0; m.ay[s] = (T)0; m.az[s] = (T)0;
        m.claim[s] = 0x7FFFFFFF;
    }
}

template <typename T>
__global__ void k_clear_sites(MdArgs<T> m)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x) {
        m.sid[s] = -1;
        m.ux[s] = kVacant; m.uy[s] = kVacant; m.uz[s] = kVacant;
        if ((void *)m.sx != (void *)m.ux) {
            m.sx[s] = (T)kVacant; m.sy[s] = (T)kVacant; m.sz[s] = (T)kVacant;
        }
        m.ax[s] = (T)0; m.ay[s] = (T)0; m.az[s] = (T)0;
        m.claim[s] = 0x7FFFFFFF;
    }
}

// Hash every atom of an explicit configuration (x: 3 natoms, A) to its
// nearest site; atoms within the skin claim the site (lowest id wins).
template <typename T>
__global__ void k_state_claim(MdArgs<T> m, const double *x, long long natoms, double Lx, double Ly, double Lz,
                              int *home, double *rel)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < natoms; i += (long long)gridDim.x * blockDim.x) {
        double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
        px -= Lx * floor(px / Lx);
        py -= Ly * floor(py / Ly);
        pz -= Lz * floor(pz / Lz);
        double rx, ry, rz;
        long long h = nearest_site(px * m.inv_half, py * m.inv_half, pz * m.inv_half, m.nx, m.ny, m.nz, rx, ry, rz);
        home[i] = (int)h;
        rel[3 * i] = rx; rel[3 * i + 1] = ry; rel[3 * i + 2] = rz;
        if (rx * rx + ry * ry + rz * rz <= m.skin2) atomicMin(&m.claim[h], (int)i);
    }
}

template <typename T>
__global__ void k_state_place(MdArgs<T> m, const double *v, long long natoms, const int *home, const double *rel)
{
    DevScalars *sc = m.sc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < natoms; i += (long long)gridDim.x * blockDim.x) {
        int h = home[i];
        double rx = rel[3 * i], ry = rel[3 * i + 1], rz = rel[3 * i + 2];
        double vx = v ? v[3 * i] : 0.0, vy = v ? v[3 * i + 1] : 0.0, vz = v ? v[3 * i + 2] : 0.0;
        if (m.claim[h] == (int)i) {
            m.sid[h] = (int)i;
            m.ux[h] = rx; m.uy[h] = ry; m.uz[h] = rz;
            if ((void *)m.sx != (void *)m.ux) {
                m.sx[h] = (T)rx; m.sy[h] = (T)ry; m.sz[h] = (T)rz;
            }
            m.vx[h] = vx; m.vy[h] = vy; m.vz[h] = vz;
        } else {
            int j = atomicAdd(&sc->n_new, 1);
            if (j < m.cap) {
                m.ra_home[j] = h;
                m.ra_id[j] = (int)i;
                m.ra_ux[j] = rx; m.ra_uy[j] = ry; m.ra_uz[j] = rz;
                m.ra_sx[j] = (T)rx; m.ra_sy[j] = (T)ry; m.ra_sz[j] = (T)rz;
                m.ra_vx[j] = vx; m.ra_vy[j] = vy; m.ra_vz[j] = vz;
                m.ra_ax[j] = (T)0; m.ra_ay[j] = (T)0; m.ra_az[j] = (T)0;
            } else {
                atomicOr(&sc->status, kStRunawayOverflow);
            }
        }
    }
}

template <typename T>
__global__ void k_set_velocities(MdArgs<T> m, const double *v)
{
    long long n = m.ns;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        int id = m.sid[s];
        if (id < 0) continue;
        m.vx[s] = v[3LL * id]; m.vy[s] = v[3LL * id + 1]; m.vz[s] = v[3LL * id + 2];
    }
    int nra = m.sc->n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        int id = m.ra_id[j];
        m.ra_vx[j] = v[3LL * id]; m.ra_vy[j] = v[3LL * id + 1]; m.ra_vz[j] = v[3LL * id + 2];
    }
}

// PKA insertion (Sec. 5.1): velocity of atom id set to speed * dir.
template <typename T>
__global__ void k_pka(MdArgs<T> m, int id, double vx, double vy, double vz)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x) {
        if (m.sid[s] == id) {
            m.vx[s] = vx; m.vy[s] = vy; m.vz[s] = vz;
        }
    }
    int nra = m.sc->n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        if (m.ra_id[j] == id) {
            m.ra_vx[j] = vx; m.ra_vy[j] = vy; m.ra_vz[j] = vz;
        }
    }
}

// max |v| over all atoms into vmax_bits (used after state changes).
template <typename T>
__global__ void k_vmax(MdArgs<T> m)
{
    double w = 0.0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x) {
        if (m.sid[s] < 0) continue;
        double v2 = m.vx[s] * m.vx[s] + m.vy[s] * m.vy[s] + m.vz[s] * m.vz[s];
        w = v2 > w ? v2 : w;
    }
    int nra = m.sc->n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        double v2 = m.ra_vx[j] * m.ra_vx[j] + m.ra_vy[j] * m.ra_vy[j] + m.ra_vz[j] * m.ra_vz[j];
        w = v2 > w ? v2 : w;
    }
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
    if ((threadIdx.x & 31) == 0 && w > 0.0)
        atomicMax(&m.sc->vmax_bits, (unsigned long long)__double_as_longlong(sqrt(w)));
}

// Per-atom read-out: kind 0 positions (A, wrapped), 1 velocities, 2 forces
// (eV/A), 3 density, 4 per-atom energy.  out is indexed by atom id.
template <typename T>
__global__ void k_scatter(MdArgs<T> m, int kind, double *out, double Lx, double Ly, double Lz)
{
    const double L[3] = {Lx, Ly, Lz};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x) {
        int id = m.sid[s];
        if (id < 0) continue;
        if (kind == 0) {
            int X, Y, Z;
            site_lat(s, m.nx, m.ny, X, Y, Z);
            double P[3] = {(X + m.ux[s]) * m.half, (Y + m.uy[s]) * m.half, (Z + m.uz[s]) * m.half};
            for (int d = 0; d < 3; ++d) out[3LL * id + d] = P[d] - L[d] * floor(P[d] / L[d]);
        } else if (kind == 1) {
            out[3LL * id] = m.vx[s]; out[3LL * id + 1] = m.vy[s]; out[3LL * id + 2] = m.vz[s];
        } else if (kind == 2) {
            out[3LL * id] = (double)m.ax[s] / m.acc_conv;
            out[3LL * id + 1] = (double)m.ay[s] / m.acc_conv;
            out[3LL * id + 2] = (double)m.az[s] / m.acc_conv;
        } else if (kind == 3) {
            out[id] = (double)m.rho[s];
        } else {
            out[id] = m.esite[s];
        }
    }
    int nra = m.sc->n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        int id = m.ra_id[j];
        if (kind == 0) {
            int X, Y, Z;
            site_lat(m.ra_home[j], m.nx, m.ny, X, Y, Z);
            double P[3] = {(X + m.ra_ux[j]) * m.half, (Y + m.ra_uy[j]) * m.half, (Z + m.ra_uz[j]) * m.half};
            for (int d = 0; d < 3; ++d) out[3LL * id + d] = P[d] - L[d] * floor(P[d] / L[d]);
        } else if (kind == 1) {
            out[3LL * id] = m.ra_vx[j]; out[3LL * id + 1] = m.ra_vy[j]; out[3LL * id + 2] = m.ra_vz[j];
        } else if (kind == 2) {
            out[3LL * id] = (double)m.ra_ax[j] / m.acc_conv;
            out[3LL * id + 1] = (double)m.ra_ay[j] / m.acc_conv;
            out[3LL * id + 2] = (double)m.ra_az[j] / m.acc_conv;
        } else if (kind == 3) {
            out[id] = (double)m.ra_rho[j];
        } else {
            out[id] = m.ra_e[j];
        }
    }
}

// Deterministic FP64 sums: potential energy (kind 0) or kinetic energy in
// amu A^2/fs^2 (kind 1) over sites and run-aways.  Stage 1 writes one
// partial per block; stage 2 (one block) adds the partials in order.
template <typename T>
__global__ void k_sum_stage1(MdArgs<T> m, int kind, double *partial)
{
    double acc = 0.0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x) {
        if (m.sid[s] < 0) continue;
        acc += kind == 0 ? m.esite[s] : (m.vx[s] * m.vx[s] + m.vy[s] * m.vy[s] + m.vz[s] * m.vz[s]);
    }
    int nra = m.sc->n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x)
        acc += kind == 0 ? m.ra_e[j] : (m.ra_vx[j] * m.ra_vx[j] + m.ra_vy[j] * m.ra_vy[j] + m.ra_vz[j] * m.ra_vz[j]);
    __shared__ double sw[32];
    acc = warp_sum<double>(acc);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_sum_stage2(const double *partial, int n, double *out)
{
    __shared__ double sw[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partial[k];
    acc = warp_sum<double>(acc);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
        *out = t;
    }
}

// Site map read-out (storage check).
template <typename T>
__global__ void k_site_map(MdArgs<T> m, long long *site_atom, long long *ra_ids)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m.ns; s += (long long)gridDim.x * blockDim.x)
        site_atom[s] = m.sid[s];
    int nra = m.sc->n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) ra_ids[j] = m.ra_id[j];
}

}  // namespace misa
