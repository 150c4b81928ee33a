// misa_newton3.cuh -- FP32 density pass with Newton's third law applied
// inside a tile (the pair-work halving of Sec. 4.2, without its write
// conflicts and without atomics).
//
// The dense shells (|n|^2 <= 12, the 58 neighbours of the crystal) are
// symmetric under n -> -n, and the shell's vectors, sorted by (z, y, x), are
// antisymmetric: v[KB + j] = -v[KE - 1 - j].  The upper half of each shell is
// the "plus" set H.  For every n in H each thread evaluates the pair
// (i, i + n) of both its sites, keeps the value for i and hands it to the
// partner i + n through a shared-memory exchange buffer indexed by tile site.
// After a barrier each site reads the value of its "minus" pair (i - n, i)
// from the buffer when i - n is a site of the tile and of the box, and
// evaluates that pair itself otherwise -- with i - n as the first site and n
// as the offset, the same operations in the same order as the thread owning
// i - n, so the value is bitwise the one that thread computes.  The density
// of a pair depends only on |r|, which is why one evaluation serves both
// sites.
//
// Per-site sums are fixed in order and independent of the tile shape: within
// a dense shell, per chunk of kN3Chunk plus offsets, the plus values in
// offset order, then the minus values in offset order; shell sums are added
// with Kahan compensation when non-zero.  Sparse shells, run-aways and the
// embedding epilogue are those of the full-neighbour pass (misa_packed.cuh).
//
// Every thread of the block runs the dense-shell loop (with its barriers);
// out-of-box and vacant sites compute harmless values and write nothing.
#pragma once

#include "misa_packed.cuh"

namespace misa {

constexpr int kN3Chunk = 4;  // plus offsets exchanged per barrier pair

// shared-memory bytes of the exchange buffer: kN3Chunk values per tile site
__host__ __device__ inline size_t n3_exchange_bytes(int tx, int ty, int tz)
{
    return sizeof(float) * kN3Chunk * 2 * (size_t)tx * ty * tz;
}

__host__ __device__ inline size_t n3_smem_bytes(size_t table_bytes, int tx, int ty, int tz, int nbuf)
{
    return ((packed_smem_bytes(table_bytes, tx, ty, tz, nbuf) + 255) & ~(size_t)255) + n3_exchange_bytes(tx, ty, tz);
}

// tile-local site index (parity, cell x, y, z over the full tile height)
template <int TX, int TY, int TZ>
__device__ __forceinline__ int n3_site(int p, int x, int y, int z)
{
    return ((p * TZ + z) * TY + y) * TX + x;
}

// a site of this tile inside the box (partial tiles at the box edge hold
// wrapped copies of other tiles' sites beyond it)
template <int TX, int TY, int TZ>
__device__ __forceinline__ bool n3_owned(const TileLoc &L, int x, int y, int z)
{
    return (unsigned)x < (unsigned)TX && (unsigned)y < (unsigned)TY && (unsigned)z < (unsigned)TZ &&
           L.c0x + x < L.rd.nx && L.c0y + y < L.rd.ny && L.c0z + z < L.rd.nz;
}

// One dense shell SH: plus pairs, exchange, minus pairs (chunks of kN3Chunk).
template <int SH, int TX, int TY, int TZ>
__device__ __forceinline__ void n3_dense_shell(const ShellInfo &shc, int seg_lo, const float4 *__restrict__ po,
                                               const float4 *__restrict__ sA,
                                               const float4 *__restrict__ sB, int slot, const PThread<TX, TY, TZ> &th,
                                               const TileLoc &L, const PairSites &ui, float2 S2, unsigned nwin,
                                               const float4 *__restrict__ tab, unsigned long long texf,
                                               float *__restrict__ xb, Acc<float> &ra, Acc<float> &rb)
{
    using G = PTile<TX, TY, TZ>;
    constexpr int KB = kLVec.shell_begin[SH], KE = kLVec.shell_begin[SH + 1];
    constexpr int HALF = (KE - KB) / 2;
    static_assert((KE - KB) % 2 == 0, "shells are symmetric");
    constexpr int NSITE = 2 * TX * TY * TZ;
    const PShell sh = pshell<SH>(shc, seg_lo);
    float2 part = make_float2(0.f, 0.f);
    const int p = th.p;
#pragma unroll 1
    for (int c0 = 0; c0 < HALF; c0 += kN3Chunk) {
        const int cn = HALF - c0 < kN3Chunk ? HALF - c0 : kN3Chunk;
        // plus pairs (i, i + n): keep, and hand to the partner
        for (int c = 0; c < cn; ++c) {
            const int k = KB + HALF + c0 + c;
            const float4 o0 = po[2 * k], o1 = po[2 * k + 1];
            const int D = __float_as_int(o1.z);
            const PGeom g = pair_geom(o0, o1, sA[slot + D], sB[slot + D], ui);
            float2 t, rs;
            int ia, ib;
            arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
            const float2 v = make_float2(cubic(tab[ia], t.x), cubic(tab_b(tab, texf, seg_lo, ib), t.y));
            part = p_add(part, v);
            const int nx = __float2int_rn(0.5f * o0.x), ny = __float2int_rn(0.5f * o0.z), nz = __float2int_rn(0.5f * o1.x);
            const int q = p ^ (nx & 1);
            const int x = th.lx + ((p + nx) >> 1), y = th.ly + ((p + ny) >> 1);
            const int za = th.lz + ((p + nz) >> 1), zb = za + G::HZ;
            if (n3_owned<TX, TY, TZ>(L, x, y, za)) xb[c * NSITE + n3_site<TX, TY, TZ>(q, x, y, za)] = v.x;
            if (n3_owned<TX, TY, TZ>(L, x, y, zb)) xb[c * NSITE + n3_site<TX, TY, TZ>(q, x, y, zb)] = v.y;
        }
        __syncthreads();
        // minus pairs (i - n, i): from the partner, or evaluated here as
        // the partner would (first site i - n, offset n)
        for (int c = 0; c < cn; ++c) {
            const int k = KB + HALF + c0 + c;
            const int km = KB + (KE - 1 - k);  // -n
            const float4 o0 = po[2 * k], o1 = po[2 * k + 1];
            const int Dm = __float_as_int(po[2 * km + 1].z);
            const int nx = __float2int_rn(0.5f * o0.x), ny = __float2int_rn(0.5f * o0.z), nz = __float2int_rn(0.5f * o1.x);
            const int x = th.lx + ((p - nx) >> 1), y = th.ly + ((p - ny) >> 1);
            const int za = th.lz + ((p - nz) >> 1), zb = za + G::HZ;
            const bool ha = n3_owned<TX, TY, TZ>(L, x, y, za), hb = n3_owned<TX, TY, TZ>(L, x, y, zb);
            float2 v;
            if (ha && hb) {
                v = make_float2(xb[c * NSITE + n3_site<TX, TY, TZ>(p, th.lx, th.ly, th.lz)],
                                xb[c * NSITE + n3_site<TX, TY, TZ>(p, th.lx, th.ly, th.lz + G::HZ)]);
            } else {
                // the partner slot (both folded sites) is the first site and
                // this thread's slot the neighbour at offset n (the 2n
                // components of a record do not depend on the parity)
                const float4 A = sA[slot + Dm], B = sB[slot + Dm];
                PairSites uj;
                uj.ux = make_float2(A.x, A.y);
                uj.uy = make_float2(A.z, A.w);
                uj.uz = make_float2(B.x, B.y);
                uj.fp = make_float2(0.f, 0.f);
                const PGeom g = pair_geom(o0, o1, sA[slot], sB[slot], uj);
                float2 t, rs;
                int ia, ib;
                arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
                v = make_float2(cubic(tab[ia], t.x), cubic(tab_b(tab, texf, seg_lo, ib), t.y));
                if (ha) v.x = xb[c * NSITE + n3_site<TX, TY, TZ>(p, th.lx, th.ly, th.lz)];
                if (hb) v.y = xb[c * NSITE + n3_site<TX, TY, TZ>(p, th.lx, th.ly, th.lz + G::HZ)];
            }
            part = p_add(part, v);
        }
        __syncthreads();
    }
    kahan_nz(ra, part.x);
    kahan_nz(rb, part.y);
}

template <int SH, int TX, int TY, int TZ>
__device__ __forceinline__ void n3_dense_shells(const ShellInfo &shc, int seg_lo, const float4 *__restrict__ po,
                                                const float4 *__restrict__ sA,
                                                const float4 *__restrict__ sB, int slot, const PThread<TX, TY, TZ> &th,
                                                const TileLoc &L, const PairSites &ui, float2 S2, unsigned nwin,
                                                const float4 *__restrict__ tab, unsigned long long texf,
                                                float *__restrict__ xb, Acc<float> &ra, Acc<float> &rb)
{
    if constexpr (SH < kSparseShell) {
        n3_dense_shell<SH, TX, TY, TZ>(shc, seg_lo, po, sA, sB, slot, th, L, ui, S2, nwin, tab, texf, xb, ra, rb);
        n3_dense_shells<SH + 1, TX, TY, TZ>(shc, seg_lo, po, sA, sB, slot, th, L, ui, S2, nwin, tab, texf, xb, ra,
                                            rb);
    }
}

template <int TX, int TY, int TZ, bool ENERGY, bool DB>
__global__ void __launch_bounds__(TX *TY *TZ, 1) k_density_n3(const __grid_constant__ GatherArgs<float> a)
{
    using G = PTile<TX, TY, TZ>;
    extern __shared__ __align__(32) unsigned char smem[];
    const int nwin = a.nseg - a.seg_lo;
    float4 *tab = reinterpret_cast<float4 *>(smem);
    for (int k = threadIdx.x; k <= nwin; k += G::NT) {
        const Vec4<float> c = k < nwin ? a.tab_f[a.seg_lo + k] : Vec4<float>{0.f, 0.f, 0.f, 0.f};
        tab[k] = make_float4(c.x, c.y, c.z, c.w);
    }
    const size_t tb = sizeof(float4) * (size_t)(nwin + 1);
    const PackedSmem sm = carve_p<TX, TY, TZ>(smem, tb, DB ? 2 : 1);
    float *xb = reinterpret_cast<float *>(smem + ((packed_smem_bytes(tb, TX, TY, TZ, DB ? 2 : 1) + 255) & ~(size_t)255));
    fill_rep_cache<float>(a, sm.rep);
    __syncthreads();

    const PThread<TX, TY, TZ> th;
    const float4 *po = &a.offp[th.p][0][0];
    const float2 S2 = p_dup(a.S);
    unsigned st = 0;
    int buf = 0;
    if constexpr (DB) {
        if ((int)blockIdx.x < a.ntiles) issue_tile_p<TX, TY, TZ, false>(a, sm.rep, sm.tA, blockIdx.x);
        cp_async_commit();
    }
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double dt_rep;
        int nra;
        const TileLoc L = locate_cached(a, sm.rep, tile, TX, TY, TZ, dt_rep, nra);
        float4 *cA = sm.tA + buf * 4 * G::PLANE;
        const float4 *cB = cA + 2 * G::PLANE;
        float U;
        if constexpr (DB) {
            const int nxt = tile + gridDim.x;
            if (nxt < a.ntiles) issue_tile_p<TX, TY, TZ, false>(a, sm.rep, sm.tA + (buf ^ 1) * 4 * G::PLANE, nxt);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            U = tile_umax_p<TX, TY, TZ, true>(cA, sm.red);
        } else {
            __syncthreads();
            U = stage_tile_p<TX, TY, TZ, false>(a, L, cA, sm.red);
        }
        const bool has_ra = a.tile_flag[tile] != 0 && nra > 0;
        const bool in_xy = (L.c0x + th.lx < L.rd.nx) && (L.c0y + th.ly < L.rd.ny);
        const bool in_a = in_xy && (L.c0z + th.lz < L.rd.nz);
        const bool in_b = in_xy && (L.c0z + th.lz + G::HZ < L.rd.nz);
        const float4 A = cA[th.slot], B = cB[th.slot];
        PairSites ui;
        ui.ux = make_float2(A.x, A.y);
        ui.uy = make_float2(A.z, A.w);
        ui.uz = make_float2(B.x, B.y);
        ui.fp = make_float2(0.f, 0.f);
        const bool live_a = in_a && A.x < 0.5f * kVacant;
        const bool live_b = in_b && A.y < 0.5f * kVacant;
        Acc<float> ra, rb;
        unsigned long long ma = 0, mb = 0;
        // dense shells: every thread (barriers inside)
        n3_dense_shells<0, TX, TY, TZ>(a.sh, a.seg_lo, po, cA, cB, th.slot, th, L, ui, S2, (unsigned)nwin, tab,
                                       a.tex_f, xb, ra, rb);
        if (live_a || live_b) {
            const float2 un = make_float2(sqrtf(A.x * A.x + A.z * A.z + B.x * B.x), sqrtf(A.y * A.y + A.w * A.w + B.y * B.y));
            const float la = a.rc_lat + un.x + U, lb = a.rc_lat + un.y + U;
            const float2 lim2 = make_float2(live_a ? la * la : -1.f, live_b ? lb * lb : -1.f);
            density_shells_p<kSparseShell>(a.sh, a.seg_lo, po, cA, cB, th.slot, ui, un, a.rc_lat, lim2, S2,
                                           (unsigned)nwin, tab, a.tex_f, ra, rb, ma, mb);
        }
        if (has_ra) {
            int pos = 0;
            const int sx = 2 * th.lx + th.p, sy = 2 * th.ly + th.p;
            const int sza = 2 * th.lz + th.p, szb = 2 * (th.lz + G::HZ) + th.p;
            const Vec4<float> ua{A.x, A.z, B.x, 0.f}, ub{A.y, A.w, B.y, 0.f};
            while (true) {
                __syncthreads();
                const int cnt = stage_runaways<float, TX, TY, TZ, false>(a, L, tile, nra, pos, sm.rh, sm.ru, sm.st);
                if (cnt == 0) break;
                if (live_a) ra_density_site(a, L, cnt, sm.rh, sm.ru, ua, sx, sy, sza, ra, st);
                if (live_b) ra_density_site(a, L, cnt, sm.rh, sm.ru, ub, sx, sy, szb, rb, st);
                if (pos >= nra) break;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const bool in = h ? in_b : in_a;
            if (!in) continue;
            const long long sid = site_of(L, th.lx, th.ly, th.lz + h * G::HZ, th.p);
            if (!(h ? live_b : live_a)) {
                a.fp_out[sid] = 0.f;
                continue;
            }
            if (a.mask_ok) a.bmask[sid] = h ? mb : ma;
            const float rh = (h ? rb : ra).value();
            float dF;
            const float Fv = embed<float>(a.tab_F, a.nseg, a.Srho, a.rho_max, rh, dF, st);
            a.fp_out[sid] = dF;
            if (ENERGY) {
                a.rho_out[sid] = rh;
                a.e_out[sid] = (double)Fv;
            }
        }
        if constexpr (DB) {
            buf ^= 1;
            __syncthreads();
        }
    }
    if constexpr (DB) cp_async_wait<0>();
    if (st) atomicOr(&a.sc[0].status, st);
}

}  // namespace misa
