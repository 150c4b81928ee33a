// misa_common.cuh -- device-side types shared by the MISA-MD GB300 kernels.
//
// Geometry convention (Sec. 3, lattice list): site (x2, cy, cz) with
// x2 in [0, 2 nx) has lattice id 2 nx ny cz + 2 nx cy + x2; p = x2 & 1 is
// the parity (0 cube corner, 1 body centre) and cx = x2 >> 1 the cell.  In
// lattice units (a0/2) the site sits at (2cx + p, 2cy + p, 2cz + p), so
// every bcc lattice vector is an integer vector whose components are all
// even or all odd.  Displacements u are stored in lattice units relative to
// the site, which makes periodic wrap implicit: a pair's separation is
// n + (u_j - u_i) with n the integer lattice vector between the two sites.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace misa {

constexpr int kMaxComp = 4;  // halo of 2 cells per axis
constexpr int kMaxN2 = 24;   // shells n^2 = 3,4,8,11,12,16,19,20,24 (136 vectors)
constexpr int kMaxShell = 16;

struct LVec {
    int x, y, z, n2;
};

constexpr bool lvec_less(const LVec &a, const LVec &b)
{
    if (a.n2 != b.n2) return a.n2 < b.n2;
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
}

constexpr int count_lvecs(int maxn2)
{
    int c = 0;
    for (int z = -kMaxComp; z <= kMaxComp; ++z)
        for (int y = -kMaxComp; y <= kMaxComp; ++y)
            for (int x = -kMaxComp; x <= kMaxComp; ++x) {
                int n2 = x * x + y * y + z * z;
                if (((x ^ y) & 1) == 0 && ((y ^ z) & 1) == 0 && n2 > 0 && n2 <= maxn2) ++c;
            }
    return c;
}

constexpr int kNVec = count_lvecs(kMaxN2);

struct LVecTable {
    LVec v[kNVec];
    int nshell;
    int shell_n2[kMaxShell];
    int shell_begin[kMaxShell + 1];
};

// All bcc lattice vectors with 0 < n^2 <= kMaxN2, sorted by (n^2, z, y, x),
// grouped into shells of equal length.
constexpr LVecTable make_lvecs()
{
    LVecTable t{};
    int c = 0;
    for (int z = -kMaxComp; z <= kMaxComp; ++z)
        for (int y = -kMaxComp; y <= kMaxComp; ++y)
            for (int x = -kMaxComp; x <= kMaxComp; ++x) {
                int n2 = x * x + y * y + z * z;
                if (((x ^ y) & 1) == 0 && ((y ^ z) & 1) == 0 && n2 > 0 && n2 <= kMaxN2) t.v[c++] = LVec{x, y, z, n2};
            }
    for (int i = 1; i < c; ++i) {
        LVec key = t.v[i];
        int j = i - 1;
        while (j >= 0 && lvec_less(key, t.v[j])) {
            t.v[j + 1] = t.v[j];
            --j;
        }
        t.v[j + 1] = key;
    }
    t.nshell = 0;
    for (int i = 0; i < c; ++i) {
        if (i == 0 || t.v[i].n2 != t.v[i - 1].n2) {
            t.shell_n2[t.nshell] = t.v[i].n2;
            t.shell_begin[t.nshell] = i;
            ++t.nshell;
        }
    }
    t.shell_begin[t.nshell] = c;
    return t;
}

constexpr LVecTable kLVec = make_lvecs();
static_assert(kNVec == 136, "bcc vectors up to n^2 = 24");

__host__ __device__ constexpr int floordiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

// Cell shift along one axis from a site of parity p along lattice component n.
__host__ __device__ constexpr int cell_shift(int p, int n) { return floordiv2(p + n); }

// Status bits (mirrors misa.h).
constexpr unsigned kStRunawayOverflow = 0x1u;
constexpr unsigned kStNonfinite = 0x2u;
constexpr unsigned kStRfloor = 0x4u;
constexpr unsigned kStRhoExtrap = 0x8u;

// A vacant site carries this displacement (lattice units): every distance
// test against it fails without a branch.
constexpr float kVacant = 1.0e4f;

// Device-resident scalars of one simulation.
struct DevScalars {
    double dt;                     // timestep of the current step
    double t;                      // simulated time
    unsigned long long vmax_bits;  // max |v| of the last completed step (double bits, >= 0)
    unsigned long long vacc_bits;  // max |v| accumulator of the running step
    long long step;
    int n_ra;       // run-away atoms in the list
    int n_ra_old;   // run-away count before this step's demotions
    int n_new;      // demotions appended this step
    int dirty;      // list needs re-sorting
    unsigned status;
    int pad;
};

// One replica (independent periodic box) of a batch.  Sites, atoms and
// run-away slots of all replicas live in pooled arrays; a replica owns the
// site range [site_base, site_base + ns), the global tiles
// [tile_base, tile_base + ntiles) and the run-away slots [ra_base, ra_base + cap).
// Atom ids equal the initial global site ids.
struct RepDesc {
    int nx, ny, nz;
    int ntx, nty, ntz;
    int ntiles, tile_base;
    long long site_base, ns;
    int ra_base, cap;
};

template <typename T>
struct alignas(2 * sizeof(T) == 8 ? 16 : 32) Vec4 {
    T x, y, z, w;
};
template <typename T>
struct alignas(2 * sizeof(T)) Vec2 {
    T x, y;
};

// Float <-> double conversions on the integer pipe (IEEE-754 binary32 /
// binary64 bit layouts).  GB300 runs FP64 (and its conversions) at a small
// fraction of the FP32 rate, while the FP64-bound integration kernels leave
// the integer pipe idle.  Both are exact for zero and every normal value
// (round to nearest even for double -> float); subnormal results flush to a
// signed zero; infinities and NaNs stay infinities and NaNs.
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    const unsigned long long mant = (unsigned long long)(b & 0x7fffffu) << 29;
    const unsigned long long ex = e == 0xffu ? 0x7ffull << 52 : (unsigned long long)(e + 896u) << 52;
    return __longlong_as_double((long long)(e == 0u ? sign : (sign | ex | mant)));
}

__device__ __forceinline__ float d2f_bits(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const unsigned e11 = (hi >> 20) & 0x7ffu;
    const int e = (int)e11 - 896;                                // binary32 biased exponent
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);       // top 23 mantissa bits
    const unsigned g = (lo >> 28) & 1u;                           // first dropped bit
    const unsigned sticky = (lo & 0x0fffffffu) != 0u ? 1u : 0u;   // any later dropped bit
    unsigned r = ((unsigned)e << 23) + m;
    r += g & (sticky | (m & 1u));  // a carry moves into the exponent (and to infinity at the top)
    if (e <= 0) r = 0u;
    if (e >= 255) r = 0x7f800000u;
    if (e11 == 0x7ffu) r = ((hi & 0xfffffu) | lo) != 0u ? 0x7fc00000u : 0x7f800000u;
    return __uint_as_float(sign | r);
}

template <typename T>
__device__ __forceinline__ Vec4<T> ld4(const Vec4<T> *p)
{
    return *p;
}

}  // namespace misa
