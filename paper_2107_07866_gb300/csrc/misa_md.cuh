// misa_md.cuh -- integration, lattice-list maintenance and read-out kernels.
//
// Velocity Verlet (Fig. 1, read as kick-drift-kick) with the adaptive
// timestep of the cascade feature list (Sec. 1), the hash update of Alg. 2
// (read with a skin: an array atom farther than skin from its site joins the
// run-away list at once; run-aways move back into empty nearest sites every
// reassign period, lowest atom id first), the run-away part of Alg. 1 (each
// run-away gathers over array sites around it and over the other
// run-aways), PKA insertion (Sec. 5.1), and per-atom read-out.
//
// Every kernel serves a whole batch of independent replicas: the replica is
// blockIdx.y (or one thread / one block per replica for the scalar and list
// kernels), and each replica has its own timestep, time and run-away list.
#pragma once

#include "misa_kernels.cuh"

namespace misa {

constexpr int kSortMax = 16384;  // run-away list capacity limit per replica (single-CTA sort)

template <typename T>
struct MdArgs {
    const RepDesc *reps;
    int nrep;
    int *sid;                      // atom id per site (pooled), -1 vacant
    double *ux, *uy, *uz;          // displacement (lattice units); vacant: kVacant
    T *sx, *sy, *sz;               // precision-T shadow of u read by the gather (aliases u in FP64)
    double *vx, *vy, *vz;
    T *ax, *ay, *az;
    T *fp, *rho;
    double *esite;
    int *claim;
    // run-away lists (pooled; replica r owns [ra_base, ra_base + cap)); the
    // home site is local to the replica; t_* is the permutation scratch
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
    int tx, ty, tz;
    DevScalars *sc;   // per replica; sc[0].status holds the batch's status bits
    double half;      // a0/2 (A per lattice unit)
    double inv_half;
    double skin2;     // skin^2, lattice units
    double dt_max, dx_max;
    int reassign_period;
    double acc_conv;  // eV/A -> A/fs^2
    double mass;
    // kick/drift blocks: block b sweeps sites [y, y + kd_chunk) of replica x
    // (block counts proportional to the replicas' sizes)
    const int2 *kd_map;
    int kd_chunk;
};

// sites per kick/drift block: 4,096 (16 per thread), fewer for a small
// handle so that its blocks still fill two waves of four CTAs per SM
constexpr int kKdChunkMax = 4096, kKdChunkMin = 512;

// local site id <-> lattice coordinates (lattice units: (2cx + p, 2cy + p, 2cz + p))
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

// the same with 32-bit divisions (a replica holds fewer than 2^31 sites),
// for the run-away pair loops; the rare paths keep the 64-bit form, whose
// division is a called routine with fewer live registers
__device__ __forceinline__ void site_lat32(int s, int nx, int ny, int &X, int &Y, int &Z)
{
    const int x2 = s % (2 * nx);
    const int r = s / (2 * nx);
    const int p = x2 & 1;
    X = x2;
    Y = 2 * (r % ny) + p;
    Z = 2 * (r / ny) + p;
}

__device__ __forceinline__ int wrapi(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// The same for a in [-n, 2n) -- a neighbour walk's cell index, whose offset
// is shorter than the box (boxes have at least 6 cells, offsets reach 4
// half-cells or 3 cells) -- by one add or subtract instead of an integer
// remainder
__device__ __forceinline__ int wrap_near(int a, int n)
{
    a += a < 0 ? n : 0;
    return a >= n ? a - n : a;
}

// The hash function of Sec. 3 in lattice units: nearest site of the point
// P (unwrapped lattice coords).  Candidates: nearest corner (all coords even)
// and nearest centre (all odd); the closer wins, a tie goes to the lower id.
// Returns the (replica-local) site id and writes P - site (lattice units).
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

// nearest_site with the site decided in FP32 wherever a margin certifies
// that the FP64 arithmetic decides the same way, FP64 otherwise: the same
// site and displacement, bit for bit, at a few FP64 operations per atom (FP64
// runs at a small fraction of the FP32 rate on GB300).  Certified when (i)
// the winning candidate's three floors are unambiguous (floor arguments
// farther from an integer than the FP32 error of P/2, so both precisions
// take the same integers) and (ii) the squared distances differ by more than
// their FP32 error plus what an ambiguous floor of the losing candidate can
// change (a coordinate of the loser then sits at distance 1 -+ 2 amb either
// way).  Bounds in units of u = 2^-24 (max |P| + 2): |fP - P| <= u per
// coordinate and |a - (P/2 + 1/2)| <= u, so a floor argument farther than
// amb = 16 u from an integer floors alike in both precisions; a squared
// distance carries <= 3 (8 u + 6 u) of FP32 rounding, and an ambiguous
// losing coordinate (P within 34 u of the tie) changes it by <= 136 u, three
// coordinates 408 u; the margin is 1024 u.
__device__ __forceinline__ long long nearest_site_fast(double Px, double Py, double Pz, int nx, int ny, int nz,
                                                       double &ux, double &uy, double &uz)
{
    const float f[3] = {d2f_bits(Px), d2f_bits(Py), d2f_bits(Pz)};
    const float pm = fmaxf(fabsf(f[0]), fmaxf(fabsf(f[1]), fabsf(f[2]))) + 2.f;
    const float amb = pm * 0x1p-20f;
    float c[3], e[3], dc = 0.f, de = 0.f;
    bool cok = true, eok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float h = 0.5f * f[d];
        const float a = h + 0.5f;
        const float fa = floorf(a), fb = floorf(h);
        cok = cok && (a - fa >= amb) && (fa + 1.f - a >= amb);
        eok = eok && (h - fb >= amb) && (fb + 1.f - h >= amb);
        c[d] = 2.f * fa;
        e[d] = fmaf(2.f, fb, 1.f);
        const float dcd = f[d] - c[d], ded = f[d] - e[d];
        dc = fmaf(dcd, dcd, dc);
        de = fmaf(ded, ded, de);
    }
    const bool corner = dc < de;
    if (fabsf(dc - de) > pm * 0x1p-14f && (corner ? cok : eok)) {
        const int X = (int)(corner ? c[0] : e[0]), Y = (int)(corner ? c[1] : e[1]), Z = (int)(corner ? c[2] : e[2]);
        ux = Px - (double)X;
        uy = Py - (double)Y;
        uz = Pz - (double)Z;
        const int cx = wrapi(X >> 1, nx), cy = wrapi(Y >> 1, ny), cz = wrapi(Z >> 1, nz);
        return (((long long)cz * ny + cy) * nx + cx) * 2 + (X & 1);
    }
    return nearest_site(Px, Py, Pz, nx, ny, nz, ux, uy, uz);
}

// grid-stride loop over the replica-local sites of replica rd
#define MISA_SITE_LOOP(rd, s)                                                                     \
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < (rd).ns;            \
         s += (long long)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// step bookkeeping (one thread per replica)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_begin_step(MdArgs<T> m)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m.nrep) return;
    DevScalars *sc = m.sc + r;
    double vmax = __longlong_as_double((long long)sc->vmax_bits);
    double dt = m.dt_max;
    if (m.dx_max > 0.0 && vmax > 0.0) dt = fmin(m.dt_max, m.dx_max / vmax);
    sc->dt = dt;
    sc->vacc_bits = 0ull;
    sc->n_ra_old = sc->n_ra;
    sc->n_new = 0;
    sc->dirty = 0;
}

// Empties the run-away bookkeeping before an explicit state is loaded (step
// count and time are kept).
template <typename T>
__global__ void k_reset_list(MdArgs<T> m)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m.nrep) return;
    DevScalars *sc = m.sc + r;
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
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m.nrep) return;
    DevScalars *sc = m.sc + r;
    sc->t += sc->dt;
    sc->step += 1;
    sc->vmax_bits = sc->vacc_bits;
}

// Opening half kick + drift of array atoms (FP64).  An atom leaving its
// skin is demoted to its replica's run-away list (Alg. 2 part 1, skin reading).
__device__ __forceinline__ double f2d(float x) { return f2d_bits(x); }
__device__ __forceinline__ double f2d(double x) { return x; }

template <typename T>
__global__ void __launch_bounds__(256, 4) k_kick_drift(MdArgs<T> m)
{
    const int2 bm = m.kd_map[blockIdx.x];
    const int r = bm.x;
    const RepDesc rd = m.reps[r];
    DevScalars *sc = m.sc + r;
    const double dt = sc->dt, hdt = 0.5 * dt, dtl = dt * m.inv_half;
    const int base = sc->n_ra_old;
    const float skin2f = (float)m.skin2;
    const long long lend = min(rd.ns, (long long)bm.y + m.kd_chunk);
    for (long long ls = bm.y + threadIdx.x; ls < lend; ls += blockDim.x) {
        const long long s = rd.site_base + ls;
        int id = m.sid[s];
        if (id < 0) continue;
        // FP64 integration; the skin test (a storage decision) in FP32;
        // FP32 <-> FP64 conversions on the integer pipe
        const double vx = fma(hdt, f2d(m.ax[s]), m.vx[s]);
        const double vy = fma(hdt, f2d(m.ay[s]), m.vy[s]);
        const double vz = fma(hdt, f2d(m.az[s]), m.vz[s]);
        const double ux = fma(dtl, vx, m.ux[s]);
        const double uy = fma(dtl, vy, m.uy[s]);
        const double uz = fma(dtl, vz, m.uz[s]);
        const float fx = d2f_bits(ux), fy = d2f_bits(uy), fz = d2f_bits(uz);
        bool out;
        if constexpr (sizeof(T) == 4) out = fx * fx + fy * fy + fz * fz > skin2f;
        else out = ux * ux + uy * uy + uz * uz > m.skin2;
        if (out) {
            int slot = atomicAdd(&sc->n_new, 1);
            int j = base + slot;
            if (j < rd.cap) {
                const int g = rd.ra_base + j;
                int X, Y, Z;
                site_lat(ls, rd.nx, rd.ny, X, Y, Z);
                double rx, ry, rz;
                long long h = nearest_site(X + ux, Y + uy, Z + uz, rd.nx, rd.ny, rd.nz, rx, ry, rz);
                m.ra_home[g] = (int)h;
                m.ra_id[g] = id;
                m.ra_ux[g] = rx; m.ra_uy[g] = ry; m.ra_uz[g] = rz;
                m.ra_sx[g] = (T)rx; m.ra_sy[g] = (T)ry; m.ra_sz[g] = (T)rz;
                m.ra_vx[g] = vx; m.ra_vy[g] = vy; m.ra_vz[g] = vz;
                m.ra_ax[g] = m.ax[s]; m.ra_ay[g] = m.ay[s]; m.ra_az[g] = m.az[s];
                m.sid[s] = -1;
                m.ux[s] = kVacant; m.uy[s] = kVacant; m.uz[s] = kVacant;
                if constexpr (sizeof(T) == 4) {
                    m.sx[s] = kVacant; m.sy[s] = kVacant; m.sz[s] = kVacant;
                }
                continue;
            }
            atomicOr(&m.sc[0].status, kStRunawayOverflow);
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
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    DevScalars *sc = m.sc + r;
    const double dt = sc->dt, hdt = 0.5 * dt;
    const int n = sc->n_ra_old;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        double vx = m.ra_vx[g] + hdt * (double)m.ra_ax[g];
        double vy = m.ra_vy[g] + hdt * (double)m.ra_ay[g];
        double vz = m.ra_vz[g] + hdt * (double)m.ra_az[g];
        int X, Y, Z;
        site_lat(m.ra_home[g], rd.nx, rd.ny, X, Y, Z);
        double Px = X + m.ra_ux[g] + dt * vx * m.inv_half;
        double Py = Y + m.ra_uy[g] + dt * vy * m.inv_half;
        double Pz = Z + m.ra_uz[g] + dt * vz * m.inv_half;
        double rx, ry, rz;
        long long h = nearest_site(Px, Py, Pz, rd.nx, rd.ny, rd.nz, rx, ry, rz);
        m.ra_home[g] = (int)h;
        m.ra_ux[g] = rx; m.ra_uy[g] = ry; m.ra_uz[g] = rz;
        m.ra_sx[g] = (T)rx; m.ra_sy[g] = (T)ry; m.ra_sz[g] = (T)rz;
        m.ra_vx[g] = vx; m.ra_vy[g] = vy; m.ra_vz[g] = vz;
    }
}

// Alg. 2 part 2: a run-away whose nearest site is empty and which lies
// within the skin of it claims the site; the lowest atom id wins.
template <typename T>
__global__ void k_reassign_claim(MdArgs<T> m, int force)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    DevScalars *sc = m.sc + r;
    if (!force && (sc->step + 1) % m.reassign_period != 0) return;
    int n = sc->n_ra_old + min(sc->n_new, rd.cap - sc->n_ra_old);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        const long long h = rd.site_base + m.ra_home[g];
        double u2 = m.ra_ux[g] * m.ra_ux[g] + m.ra_uy[g] * m.ra_uy[g] + m.ra_uz[g] * m.ra_uz[g];
        if (m.sid[h] < 0 && u2 <= m.skin2) {
            atomicMin(&m.claim[h], m.ra_id[g]);
            sc->dirty = 1;
        }
    }
}

template <typename T>
__global__ void k_reassign_promote(MdArgs<T> m, int force)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    DevScalars *sc = m.sc + r;
    if (!force && (sc->step + 1) % m.reassign_period != 0) return;
    int n = sc->n_ra_old + min(sc->n_new, rd.cap - sc->n_ra_old);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        const long long h = rd.site_base + m.ra_home[g];
        int id = m.ra_id[g];
        if (m.claim[h] == id && m.sid[h] < 0) {
            m.sid[h] = id;
            m.ux[h] = m.ra_ux[g]; m.uy[h] = m.ra_uy[g]; m.uz[h] = m.ra_uz[g];
            if constexpr (sizeof(T) == 4) {
                m.sx[h] = (T)m.ra_ux[g]; m.sy[h] = (T)m.ra_uy[g]; m.sz[h] = (T)m.ra_uz[g];
            }
            m.vx[h] = m.ra_vx[g]; m.vy[h] = m.ra_vy[g]; m.vz[h] = m.ra_vz[g];
            m.ax[h] = m.ra_ax[g]; m.ay[h] = m.ra_ay[g]; m.az[h] = m.ra_az[g];
            m.ra_id[g] = -1;  // removed from the list by k_ra_sort
        }
    }
}

// Rebuilds each replica's run-away list in ascending atom id (deterministic
// order for every gather that scans it), dropping promoted entries; resets
// the site claims.  One CTA per replica, bitonic sort of (id, index) keys in
// shared memory.
template <typename T>
__global__ void __launch_bounds__(1024) k_ra_sort(MdArgs<T> m)
{
    extern __shared__ unsigned long long skey[];
    __shared__ int s_cnt;
    const int r = blockIdx.x;
    const RepDesc rd = m.reps[r];
    DevScalars *sc = m.sc + r;
    const int nnew = sc->n_new;
    const int n = sc->n_ra_old + min(nnew, rd.cap - sc->n_ra_old);
    if (nnew == 0 && sc->dirty == 0) return;
    const int B = rd.ra_base;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned long long key = ~0ull;
        if (i < n) {
            int id = m.ra_id[B + i];
            key = ((unsigned long long)(id < 0 ? 0xFFFFFFFFu : (unsigned)id) << 32) | (unsigned)i;
            m.claim[rd.site_base + m.ra_home[B + i]] = 0x7FFFFFFF;
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
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int local = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if ((skey[i] >> 32) != 0xFFFFFFFFull) ++local;
    atomicAdd(&s_cnt, local);
    __syncthreads();
    const int cnt = s_cnt;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int src = B + (int)(skey[i] & 0xFFFFFFFFu), d = B + i;
        m.t_home[d] = m.ra_home[src];
        m.t_id[d] = m.ra_id[src];
        m.t_u[0][d] = m.ra_ux[src]; m.t_u[1][d] = m.ra_uy[src]; m.t_u[2][d] = m.ra_uz[src];
        m.t_v[0][d] = m.ra_vx[src]; m.t_v[1][d] = m.ra_vy[src]; m.t_v[2][d] = m.ra_vz[src];
        m.t_s[0][d] = m.ra_sx[src]; m.t_s[1][d] = m.ra_sy[src]; m.t_s[2][d] = m.ra_sz[src];
        m.t_a[0][d] = m.ra_ax[src]; m.t_a[1][d] = m.ra_ay[src]; m.t_a[2][d] = m.ra_az[src];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int d = B + i;
        m.ra_home[d] = m.t_home[d];
        m.ra_id[d] = m.t_id[d];
        m.ra_ux[d] = m.t_u[0][d]; m.ra_uy[d] = m.t_u[1][d]; m.ra_uz[d] = m.t_u[2][d];
        m.ra_vx[d] = m.t_v[0][d]; m.ra_vy[d] = m.t_v[1][d]; m.ra_vz[d] = m.t_v[2][d];
        m.ra_sx[d] = m.t_s[0][d]; m.ra_sy[d] = m.t_s[1][d]; m.ra_sz[d] = m.t_s[2][d];
        m.ra_ax[d] = m.t_a[0][d]; m.ra_ay[d] = m.t_a[1][d]; m.ra_az[d] = m.t_a[2][d];
    }
    if (threadIdx.x == 0) {
        sc->n_ra = cnt;
        if (sc->n_ra_old + nnew > rd.cap) atomicOr(&m.sc[0].status, kStRunawayOverflow);
    }
}

// ---------------------------------------------------------------------------
// per-tile run-away index (the "run-away bucket" of every tile of a map)
// ---------------------------------------------------------------------------
// A tile stages the run-aways whose home cell lies within 3 cells of it
// (ra_in_tile).  Rather than every tile scanning the whole list, each tile
// gets the sorted list indices of its run-aways: count (atomics), segment
// allocation, fill (atomics), then a per-tile sort restores list order, so
// a tile stages exactly the entries, in exactly the order, the scan would.
// tile_flag: 0 no run-away, 1 indexed, 2 scan the list (the index ran out
// of room or a segment is too long to sort).

constexpr int kRaSortSeg = 1024;  // longest segment a warp sorts

struct RaTileMap {
    const RepDesc *reps;  // the map's replica table (tile counts of its shape)
    int tx, ty, tz;
    int ntiles;
    int *flag, *cnt, *off, *fill, *list;
    int *nz;     // tiles with run-aways (compact)
    int *aux;    // [0] segment cursor, [1] nz count
    int cap;     // list entries
};

// The distinct tiles along one axis that hold a cell within 3 of cell c
// (periodic, the whole axis for boxes under 7 cells), kept in registers (no
// local-memory arrays).  Tiles have 4 or more cells, so the 7-cell window
// meets at most four: two across the wrap (a partial last tile and the one
// before it) and two from cell 0 on.
struct AxisTiles {
    int t0, t1, t2, t3, n;
};

__device__ __forceinline__ AxisTiles axis_tiles(int c, int nn, int tt)
{
    AxisTiles r{-1, -1, -1, -1, 0};
    const int w = nn < 7 ? nn : 7;
    for (int o = 0; o < w; ++o) {
        const int t = wrap_near(c - 3 + o, nn) / tt;
        if (t == r.t0 || t == r.t1 || t == r.t2 || t == r.t3) continue;
        if (r.n == 0) r.t0 = t;
        else if (r.n == 1) r.t1 = t;
        else if (r.n == 2) r.t2 = t;
        else r.t3 = t;
        ++r.n;
    }
    return r;
}

__device__ __forceinline__ int axis_tile(const AxisTiles &a, int k)
{
    return k == 0 ? a.t0 : (k == 1 ? a.t1 : (k == 2 ? a.t2 : a.t3));
}

// calls f(global tile, tile coords) for every tile of rd within 3 cells of
// the home cell of site h (a superset of the tiles that stage the run-away
// for small boxes; exactly those when every axis has tile + 6 cells or more)
template <typename F>
__device__ __forceinline__ void for_ra_tiles(const RepDesc &rd, int h, int tx, int ty, int tz, F f)
{
    const int x2 = h % (2 * rd.nx);
    const int q = h / (2 * rd.nx);
    const AxisTiles ax = axis_tiles(x2 >> 1, rd.nx, tx), ay = axis_tiles(q % rd.ny, rd.ny, ty),
                    az = axis_tiles(q / rd.ny, rd.nz, tz);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        if (a >= az.n) break;
        const int tiz = axis_tile(az, a);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (b >= ay.n) break;
            const int tiy = axis_tile(ay, b);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (e >= ax.n) break;
                const int tix = axis_tile(ax, e);
                f(rd.tile_base + (tiz * rd.nty + tiy) * rd.ntx + tix, tix, tiy, tiz);
            }
        }
    }
}

// the stage predicate of tile (tix, tiy, tiz) of a tx x ty x tz map (the
// enumeration above is a superset for small boxes)
__device__ __forceinline__ bool ra_takes_rt(const RepDesc &rd, int h, int tx, int ty, int tz, int tix, int tiy, int tiz)
{
    int hx, hy, hz;
    return ra_in_tile_rt(rd, h, tix * tx, tiy * ty, tiz * tz, tx, ty, tz, hx, hy, hz);
}

struct RaTileMaps {
    RaTileMap m[2];  // density pass's map, force pass's map
};

// The tiles of map M that stage a run-away with home site h: the
// enumeration, filtered by the stage predicate where a box is too small for
// the two to agree (an axis of fewer than tile + 6 cells).
template <typename F>
__device__ __forceinline__ void for_staging_tiles(const RepDesc &rd, const RaTileMap &M, int h, F f)
{
    const bool exact = rd.nx >= M.tx + 6 && rd.ny >= M.ty + 6 && rd.nz >= M.tz + 6;
    for_ra_tiles(rd, h, M.tx, M.ty, M.tz, [&](int t, int tix, int tiy, int tiz) {
        if (exact || ra_takes_rt(rd, h, M.tx, M.ty, M.tz, tix, tiy, tiz)) f(t);
    });
}

// grid.y = replica; both maps
template <typename T>
__global__ void k_ra_tcount(MdArgs<T> m, RaTileMaps Ms)
{
    const int r = blockIdx.y;
    const int n = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const RaTileMap &M = Ms.m[k];
            const RepDesc rd = M.reps[r];
            for_staging_tiles(rd, M, m.ra_home[rd.ra_base + j], [&](int t) { atomicAdd(&M.cnt[t], 1); });
        }
    }
}

// segment of every tile with run-aways; its flag; the fill cursors reset
static __global__ void k_ra_toff(RaTileMaps Ms)
{
    for (int k = 0; k < 2; ++k) {
        const RaTileMap &M = Ms.m[k];
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M.ntiles; t += gridDim.x * blockDim.x) {
            const int c = M.cnt[t];
            int flag = 0;
            if (c > 0) {
                const int o = atomicAdd(&M.aux[0], c);
                M.off[t] = o;
                flag = (o + c <= M.cap && c <= kRaSortSeg) ? 1 : 2;
                if (flag == 1 && c > 1) M.nz[atomicAdd(&M.aux[1], 1)] = t;
            }
            M.flag[t] = flag;
            M.fill[t] = 0;
        }
    }
}

template <typename T>
__global__ void k_ra_tfill(MdArgs<T> m, RaTileMaps Ms)
{
    const int r = blockIdx.y;
    const int n = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const RaTileMap &M = Ms.m[k];
            const RepDesc rd = M.reps[r];
            for_staging_tiles(rd, M, m.ra_home[rd.ra_base + j], [&](int t) {
                if (M.flag[t] == 1) M.list[M.off[t] + atomicAdd(&M.fill[t], 1)] = j;
            });
        }
    }
}

// one warp per tile with two or more entries: bitonic sort of its segment
// in shared memory (ascending list index = list order)
constexpr int kRaSortWarps = 4;
static __global__ void __launch_bounds__(32 * kRaSortWarps) k_ra_tsort(RaTileMaps Ms)
{
    __shared__ int buf[kRaSortWarps][kRaSortSeg];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *b = buf[w];
    const RaTileMap &M = Ms.m[blockIdx.y];
    const int nz = M.aux[1];
    for (int q = blockIdx.x * kRaSortWarps + w; q < nz; q += gridDim.x * kRaSortWarps) {
        const int t = M.nz[q];
        const int c = M.cnt[t], o = M.off[t];
        int P = 32;
        while (P < c) P <<= 1;
        for (int i = lane; i < P; i += 32) b[i] = i < c ? M.list[o + i] : 0x7FFFFFFF;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const int x = b[i], y = b[l];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) {
                            b[i] = y;
                            b[l] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < c; i += 32) M.list[o + i] = b[i];
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// run-away gather (Alg. 1 parts 2-3): one warp per run-away atom
// ---------------------------------------------------------------------------

template <typename T>
struct RaGatherArgs {
    GatherArgs<T> g;  // tables, replica table, site arrays
    const int *sid;
    const T *ra_sx, *ra_sy, *ra_sz;
    T *ra_fp, *ra_rho;
    double *ra_e;
    T *ra_ax, *ra_ay, *ra_az;
    double *ra_vx, *ra_vy, *ra_vz;
    int energy;
    int tx, ty, tz;  // tile shape of g's map (its per-tile run-away index)
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kRaBatch = 4;  // window sites a lane loads at once

// mode 0: density (+F, F'), mode 1: force (+kick); grid.y = replica
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_ra_gather(const __grid_constant__ RaGatherArgs<T> ra)
{
    const GatherArgs<T> &a = ra.g;
    const int rep = blockIdx.y;
    const RepDesc rd = a.reps[rep];
    DevScalars *scr = a.sc + rep;
    const int n = scr->n_ra;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const double hdt = 0.5 * scr->dt;
    const int B = rd.ra_base;
    unsigned st = 0;
    double vmax2 = 0.0;
    const int Lx = 2 * rd.nx, Ly = 2 * rd.ny, Lz = 2 * rd.nz;
    for (int j = warp; j < n; j += nwarps) {
        int h = a.ra_home[B + j];
        int X, Y, Z;
        site_lat32(h, rd.nx, rd.ny, X, Y, Z);
        const int hp = X & 1;
        const int hcx = X >> 1, hcy = (Y - hp) >> 1, hcz = (Z - hp) >> 1;
        T ujx = ra.ra_sx[B + j], ujy = ra.ra_sy[B + j], ujz = ra.ra_sz[B + j];
        T fpj = MODE == 1 ? ra.ra_fp[B + j] : (T)0;
        Acc<T> s0, s1, s2;
        double ephi = 0.0;
        const int wx = rd.nx < 7 ? rd.nx : 7, wy = rd.ny < 7 ? rd.ny : 7, wz = rd.nz < 7 ? rd.nz : 7;
        const int W = wx * wy * wz * 2;
        // lane l takes the window's sites c = l, l + 32, ... in ascending
        // order; kRaBatch of them at a time, each dependent load (site id,
        // displacement, table segment) issued for the whole batch before the
        // next, so the chain of load latencies is W / (32 kRaBatch) batches
        // long rather than W / 32 sites
        for (int c0 = lane; c0 < W; c0 += 32 * kRaBatch) {
            long long sb[kRaBatch];
            bool ok[kRaBatch];
            int nb[kRaBatch][3];
#pragma unroll
            for (int b = 0; b < kRaBatch; ++b) {
                const int c = c0 + 32 * b;
                const int q = c & 1;
                const int rr = c >> 1;
                const int ox = rr % wx, oy = (rr / wx) % wy, oz = rr / (wx * wy);
                const int cx = hcx - 3 + ox, cy = hcy - 3 + oy, cz = hcz - 3 + oz;
                sb[b] = rd.site_base +
                        (((long long)wrap_near(cz, rd.nz) * rd.ny + wrap_near(cy, rd.ny)) * rd.nx + wrap_near(cx, rd.nx)) * 2 + q;
                nb[b][0] = 2 * cx + q - X; nb[b][1] = 2 * cy + q - Y; nb[b][2] = 2 * cz + q - Z;
                ok[b] = c < W && ra.sid[c < W ? sb[b] : rd.site_base] >= 0;
            }
            T dxb[kRaBatch], dyb[kRaBatch], dzb[kRaBatch], fpb[kRaBatch];
#pragma unroll
            for (int b = 0; b < kRaBatch; ++b) {
                const long long s = ok[b] ? sb[b] : rd.site_base;
                dxb[b] = a.ux[s] - ujx; dyb[b] = a.uy[s] - ujy; dzb[b] = a.uz[s] - ujz;
                fpb[b] = MODE == 1 ? a.fp[s] : (T)0;
            }
            int segb[kRaBatch];
            T tb[kRaBatch], rinvb[kRaBatch];
            bool inb[kRaBatch], fhb[kRaBatch];
#pragma unroll
            for (int b = 0; b < kRaBatch; ++b) {
                const T dx = dxb[b], dy = dyb[b], dz = dzb[b];
                const int nx_ = nb[b][0], ny_ = nb[b][1], nz_ = nb[b][2];
                T qq = (dx + (T)(2 * nx_)) * dx + (dy + (T)(2 * ny_)) * dy + (dz + (T)(2 * nz_)) * dz;
                T r2 = (T)(nx_ * nx_ + ny_ * ny_ + nz_ * nz_) + qq;
                inb[b] = ok[b] && r2 < a.rc2;
                direct_arg<T>(inb[b] ? r2 : a.rfloor2, a.S, a.rfloor2, segb[b], tb[b], rinvb[b], fhb[b]);
                segb[b] = clamp_seg<T>(segb[b], a.nseg, tb[b]);
            }
#pragma unroll
            for (int b = 0; b < kRaBatch; ++b) {
                if (!inb[b]) continue;
                const int seg = segb[b];
                const T t = tb[b];
                const bool fh = fhb[b];
                if (fh) st |= kStRfloor;
                if (MODE == 0) {
                    Vec4<T> cf = a.tab_f[seg];
                    s0.add(((cf.x * t + cf.y) * t + cf.z) * t + cf.w);
                } else {
                    Vec4<T> c0 = a.tab_d0[seg];
                    Vec2<T> c1 = a.tab_d1[seg];
                    T dfr = (c0.x * t + c0.y) * t + c0.z;
                    T dph = (c0.w * t + c1.x) * t + c1.y;
                    T coef = (fpj + fpb[b]) * dfr + dph;
                    T sc = fh ? (T)0 : coef * rinvb[b];
                    s0.add(sc * (dxb[b] + (T)nb[b][0]));
                    s1.add(sc * (dyb[b] + (T)nb[b][1]));
                    s2.add(sc * (dzb[b] + (T)nb[b][2]));
                    if (ra.energy) {
                        Vec4<T> cp = a.tab_phi[seg];
                        ephi += 0.5 * (double)(((cp.x * t + cp.y) * t + cp.z) * t + cp.w);
                    }
                }
            }
        }
        // the other run-aways: those of the home tile's index entry (every
        // run-away within rc of this one is among them) when the list is
        // longer than kRaScanMax, else the whole list; either way lane l
        // takes the list indices k = l mod 32 in ascending order, so the
        // sums do not depend on the index
        const int tix = hcx / ra.tx, tiy = hcy / ra.ty, tiz = hcz / ra.tz;
        const int tl = rd.tile_base + (tiz * rd.nty + tiy) * rd.ntx + tix;
        const bool indexed = n > kRaScanMax && a.tile_flag[tl] == 1;
        const int nk = indexed ? a.ra_tcnt[tl] : (n + 31 - lane) / 32;
        const int *klist = indexed ? a.ra_tlist + a.ra_toff[tl] : nullptr;
        for (int kq = 0; kq < nk; ++kq) {
            const int k = indexed ? klist[kq] : lane + 32 * kq;
            if (indexed && (k & 31) != lane) continue;
            if (k == j) continue;
            int Xk, Yk, Zk;
            site_lat32(a.ra_home[B + k], rd.nx, rd.ny, Xk, Yk, Zk);
            int nx_ = Xk - X, ny_ = Yk - Y, nz_ = Zk - Z;
            nx_ -= (nx_ > rd.nx) ? Lx : 0;
            nx_ += (nx_ < -rd.nx) ? Lx : 0;
            ny_ -= (ny_ > rd.ny) ? Ly : 0;
            ny_ += (ny_ < -rd.ny) ? Ly : 0;
            nz_ -= (nz_ > rd.nz) ? Lz : 0;
            nz_ += (nz_ < -rd.nz) ? Lz : 0;
            T dx = ra.ra_sx[B + k] - ujx, dy = ra.ra_sy[B + k] - ujy, dz = ra.ra_sz[B + k] - ujz;
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
                    T coef = (fpj + ra.ra_fp[B + k]) * dfr + dph;
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
                ra.ra_fp[B + j] = dF;
                if (ra.energy) {
                    ra.ra_rho[B + j] = rh;
                    ra.ra_e[B + j] = (double)Fv;
                }
            }
        } else {
            T fx = warp_sum<T>(s0.value()), fy = warp_sum<T>(s1.value()), fz = warp_sum<T>(s2.value());
            double eph = warp_sum<double>(ephi);
            if (lane == 0) {
                double conv = a.acc_conv;
                double gx = (double)fx * conv, gy = (double)fy * conv, gz = (double)fz * conv;
                ra.ra_ax[B + j] = (T)gx;
                ra.ra_ay[B + j] = (T)gy;
                ra.ra_az[B + j] = (T)gz;
                if (!isfinite(gx) || !isfinite(gy) || !isfinite(gz)) st |= kStNonfinite;
                if (a.kick) {
                    double vx = ra.ra_vx[B + j] + hdt * (double)(T)gx;
                    double vy = ra.ra_vy[B + j] + hdt * (double)(T)gy;
                    double vz = ra.ra_vz[B + j] + hdt * (double)(T)gz;
                    ra.ra_vx[B + j] = vx;
                    ra.ra_vy[B + j] = vy;
                    ra.ra_vz[B + j] = vz;
                    double v2 = vx * vx + vy * vy + vz * vz;
                    vmax2 = v2 > vmax2 ? v2 : vmax2;
                }
                if (ra.energy) ra.ra_e[B + j] += eph;
            }
        }
    }
    if (st) atomicOr(&a.sc[0].status, st);
    if (MODE == 1 && a.kick && lane == 0 && vmax2 > 0.0)
        atomicMax(&scr->vacc_bits, (unsigned long long)__double_as_longlong(sqrt(vmax2)));
}

// ---------------------------------------------------------------------------
// state set-up and read-out (grid.y = replica)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_init_crystal(MdArgs<T> m)
{
    const RepDesc rd = m.reps[blockIdx.y];
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        m.sid[s] = (int)s;
        m.ux[s] = 0.0; m.uy[s] = 0.0; m.uz[s] = 0.0;
        if constexpr (sizeof(T) == 4) {
            m.sx[s] = 0.f; m.sy[s] = 0.f; m.sz[s] = 0.f;
        }
        m.vx[s] = 0.0; m.vy[s] = 0.0; m.vz[s] = 0.0;
        m.ax[s] = (T)0; m.ay[s] = (T)0; m.az[s] = (T)0;
        m.claim[s] = 0x7FFFFFFF;
    }
}

template <typename T>
__global__ void k_clear_sites(MdArgs<T> m)
{
    const RepDesc rd = m.reps[blockIdx.y];
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        m.sid[s] = -1;
        m.ux[s] = kVacant; m.uy[s] = kVacant; m.uz[s] = kVacant;
        if constexpr (sizeof(T) == 4) {
            m.sx[s] = kVacant; m.sy[s] = kVacant; m.sz[s] = kVacant;
        }
        m.ax[s] = (T)0; m.ay[s] = (T)0; m.az[s] = (T)0;
        m.claim[s] = 0x7FFFFFFF;
    }
}

// Hash every atom of an explicit configuration (x: 3 natoms, A) to the
// nearest site of its replica's box; atoms within the skin claim the site
// (lowest id wins).  Atom i of replica r is i in [site_base, site_base + ns).
template <typename T>
__global__ void k_state_claim(MdArgs<T> m, const double *x, int *home, double *rel)
{
    const RepDesc rd = m.reps[blockIdx.y];
    const double L[3] = {rd.nx * 2.0 * m.half, rd.ny * 2.0 * m.half, rd.nz * 2.0 * m.half};
    // p - L floor(p / L) leaves p in [0, L (1 - 2^-50)) unchanged (the
    // quotient stays below 1): only other coordinates take the division.
    // Non-negative doubles order as their bit patterns (integer compares).
    long long Lw[3];
    for (int d = 0; d < 3; ++d) Lw[d] = __double_as_longlong(L[d] * (1.0 - 0x1p-50));
    MISA_SITE_LOOP(rd, li) {
        const long long i = rd.site_base + li;
        double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const long long b = __double_as_longlong(p[d]);
            if (b < 0 || b >= Lw[d]) p[d] -= L[d] * floor(p[d] / L[d]);
        }
        double rx, ry, rz;
        long long h = nearest_site_fast(p[0] * m.inv_half, p[1] * m.inv_half, p[2] * m.inv_half, rd.nx, rd.ny, rd.nz,
                                        rx, ry, rz);
        home[i] = (int)h;
        rel[3 * i] = rx; rel[3 * i + 1] = ry; rel[3 * i + 2] = rz;
        if (rx * rx + ry * ry + rz * rz <= m.skin2) atomicMin(&m.claim[rd.site_base + h], (int)i);
    }
}

template <typename T>
__global__ void k_state_place(MdArgs<T> m, const double *v, const int *home, const double *rel)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    DevScalars *sc = m.sc + r;
    MISA_SITE_LOOP(rd, li) {
        const long long i = rd.site_base + li;
        const int h = home[i];
        const long long hs = rd.site_base + h;
        double rx = rel[3 * i], ry = rel[3 * i + 1], rz = rel[3 * i + 2];
        double vx = v ? v[3 * i] : 0.0, vy = v ? v[3 * i + 1] : 0.0, vz = v ? v[3 * i + 2] : 0.0;
        if (m.claim[hs] == (int)i) {
            m.sid[hs] = (int)i;
            m.ux[hs] = rx; m.uy[hs] = ry; m.uz[hs] = rz;
            if constexpr (sizeof(T) == 4) {
                m.sx[hs] = (T)rx; m.sy[hs] = (T)ry; m.sz[hs] = (T)rz;
            }
            m.vx[hs] = vx; m.vy[hs] = vy; m.vz[hs] = vz;
        } else {
            int j = atomicAdd(&sc->n_new, 1);
            if (j < rd.cap) {
                const int g = rd.ra_base + j;
                m.ra_home[g] = h;
                m.ra_id[g] = (int)i;
                m.ra_ux[g] = rx; m.ra_uy[g] = ry; m.ra_uz[g] = rz;
                m.ra_sx[g] = (T)rx; m.ra_sy[g] = (T)ry; m.ra_sz[g] = (T)rz;
                m.ra_vx[g] = vx; m.ra_vy[g] = vy; m.ra_vz[g] = vz;
                m.ra_ax[g] = (T)0; m.ra_ay[g] = (T)0; m.ra_az[g] = (T)0;
            } else {
                atomicOr(&m.sc[0].status, kStRunawayOverflow);
            }
        }
    }
}

template <typename T>
__global__ void k_set_velocities(MdArgs<T> m, const double *v)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        int id = m.sid[s];
        if (id < 0) continue;
        m.vx[s] = v[3LL * id]; m.vy[s] = v[3LL * id + 1]; m.vz[s] = v[3LL * id + 2];
    }
    int nra = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        int id = m.ra_id[g];
        m.ra_vx[g] = v[3LL * id]; m.ra_vy[g] = v[3LL * id + 1]; m.ra_vz[g] = v[3LL * id + 2];
    }
}

// PKA insertion (Sec. 5.1): velocity of atom id set to speed * dir.
template <typename T>
__global__ void k_pka(MdArgs<T> m, int id, double vx, double vy, double vz)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        if (m.sid[s] == id) {
            m.vx[s] = vx; m.vy[s] = vy; m.vz[s] = vz;
        }
    }
    int nra = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        if (m.ra_id[g] == id) {
            m.ra_vx[g] = vx; m.ra_vy[g] = vy; m.ra_vz[g] = vz;
        }
    }
}

// max |v| of every replica into its vmax_bits (used after state changes).
template <typename T>
__global__ void k_vmax(MdArgs<T> m)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    double w = 0.0;
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        if (m.sid[s] < 0) continue;
        double v2 = m.vx[s] * m.vx[s] + m.vy[s] * m.vy[s] + m.vz[s] * m.vz[s];
        w = v2 > w ? v2 : w;
    }
    int nra = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        double v2 = m.ra_vx[g] * m.ra_vx[g] + m.ra_vy[g] * m.ra_vy[g] + m.ra_vz[g] * m.ra_vz[g];
        w = v2 > w ? v2 : w;
    }
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
    if ((threadIdx.x & 31) == 0 && w > 0.0)
        atomicMax(&m.sc[r].vmax_bits, (unsigned long long)__double_as_longlong(sqrt(w)));
}

// Per-atom read-out: kind 0 positions (A, wrapped into the replica's box),
// 1 velocities, 2 forces (eV/A), 3 density, 4 per-atom energy.  out is
// indexed by atom id.
template <typename T>
__global__ void k_scatter(MdArgs<T> m, int kind, double *out)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    const double L[3] = {rd.nx * 2.0 * m.half, rd.ny * 2.0 * m.half, rd.nz * 2.0 * m.half};
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        int id = m.sid[s];
        if (id < 0) continue;
        if (kind == 0) {
            int X, Y, Z;
            site_lat(ls, rd.nx, rd.ny, X, Y, Z);
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
    int nra = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        int id = m.ra_id[g];
        if (kind == 0) {
            int X, Y, Z;
            site_lat(m.ra_home[g], rd.nx, rd.ny, X, Y, Z);
            double P[3] = {(X + m.ra_ux[g]) * m.half, (Y + m.ra_uy[g]) * m.half, (Z + m.ra_uz[g]) * m.half};
            for (int d = 0; d < 3; ++d) out[3LL * id + d] = P[d] - L[d] * floor(P[d] / L[d]);
        } else if (kind == 1) {
            out[3LL * id] = m.ra_vx[g]; out[3LL * id + 1] = m.ra_vy[g]; out[3LL * id + 2] = m.ra_vz[g];
        } else if (kind == 2) {
            out[3LL * id] = (double)m.ra_ax[g] / m.acc_conv;
            out[3LL * id + 1] = (double)m.ra_ay[g] / m.acc_conv;
            out[3LL * id + 2] = (double)m.ra_az[g] / m.acc_conv;
        } else if (kind == 3) {
            out[id] = (double)m.ra_rho[g];
        } else {
            out[id] = m.ra_e[g];
        }
    }
}

// Deterministic FP64 sums per replica: potential energy (kind 0) or sum of
// |v|^2 (kind 1) over sites and run-aways.  Stage 1 writes one partial per
// (replica, block); stage 2 (one block per replica) adds them in order.
template <typename T>
__global__ void k_sum_stage1(MdArgs<T> m, int kind, double *partial)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    double acc = 0.0;
    MISA_SITE_LOOP(rd, ls) {
        const long long s = rd.site_base + ls;
        if (m.sid[s] < 0) continue;
        acc += kind == 0 ? m.esite[s] : (m.vx[s] * m.vx[s] + m.vy[s] * m.vy[s] + m.vz[s] * m.vz[s]);
    }
    int nra = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x) {
        const int g = rd.ra_base + j;
        acc += kind == 0 ? m.ra_e[g] : (m.ra_vx[g] * m.ra_vx[g] + m.ra_vy[g] * m.ra_vy[g] + m.ra_vz[g] * m.ra_vz[g]);
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

static __global__ void k_sum_stage2(const double *partial, int n, double *out)
{
    __shared__ double sw[32];
    const double *pr = partial + (size_t)blockIdx.x * n;
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += pr[k];
    acc = warp_sum<double>(acc);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
        out[blockIdx.x] = t;
    }
}

// Site map read-out (storage check): atom per site; run-away ids at their
// pooled slots.
// Wigner-Seitz defect count (the vacancies and interstitials behind the
// Frenkel-pair curves of Sec. 5.1).  An array atom lies within the skin of
// its own site, so it belongs to that site's cell; a run-away belongs to its
// home, its nearest site.  Atoms = sites, so vacancies = interstitials =
// run-aways - (distinct empty sites that are the home of a run-away).
// k_defects_reset marks every run-away home; k_defects_count claims each
// empty home once.  grid.y = replica.
template <typename T>
__global__ void k_defects_reset(MdArgs<T> m, int *mark)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    const int n = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        mark[rd.site_base + m.ra_home[rd.ra_base + j]] = -1;
}

template <typename T>
__global__ void k_defects_count(MdArgs<T> m, int *mark, unsigned long long *filled)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    const int n = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const long long h = rd.site_base + m.ra_home[rd.ra_base + j];
        if (m.sid[h] < 0 && atomicCAS(&mark[h], -1, j) == -1) atomicAdd(&filled[r], 1ull);
    }
}

template <typename T>
__global__ void k_site_map(MdArgs<T> m, long long *site_atom, long long *ra_ids)
{
    const int r = blockIdx.y;
    const RepDesc rd = m.reps[r];
    MISA_SITE_LOOP(rd, ls) site_atom[rd.site_base + ls] = m.sid[rd.site_base + ls];
    int nra = m.sc[r].n_ra;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nra; j += gridDim.x * blockDim.x)
        ra_ids[rd.ra_base + j] = m.ra_id[rd.ra_base + j];
}

}  // namespace misa
