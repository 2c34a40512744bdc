// Device-side data layout and per-node arithmetic of the D2Q9 pseudopotential
// MRT step (Shan et al., arXiv:1605.01800, Sec. 2).
//
// Layout in HBM (one array per ping-pong buffer, all lattices of a batch):
//   lattice L owns 9 planes starting at element geom[L].f_off; plane a holds
//   f_a (or its deviation f_a - w_a rho_ref) at element a*plane + idx(x, y),
//   idx(x, y) = (y + kGY) * pitch + x + kGX. kGX = 32 keeps node x = 0 (and
//   every row's first node) on a 128-byte boundary; pitch = round_up(nx + 34,
//   32). The frame around the nodes (kGY rows above and below, the columns
//   left and right of them) holds no populations: periodic streaming wraps
//   by address arithmetic (Nbr below), so a step reads and writes only the
//   nodes themselves, 9 + 9 populations each, with no copies of edge nodes
//   to keep in step. The frame gives the read-out's psi plane room for its
//   one-cell halo. The wall mask uses the same idx() (one byte per cell; its
//   frame holds the periodic images, written once by the host).
//
// Velocity numbering (weights of Eq. 7: axis 1-4, diagonal 5-8):
//   e0 (0,0) e1 (1,0) e2 (0,1) e3 (-1,0) e4 (0,-1)
//   e5 (1,1) e6 (-1,1) e7 (-1,-1) e8 (1,-1)
// Moment order (Eq. 4): rho, e, zeta, j_x, q_x, j_y, q_y, p_xx, p_xy.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr unsigned FLAG_PSI_CLAMPED = 1u;
constexpr unsigned FLAG_NONFINITE = 2u;
constexpr unsigned FLAG_TIMEOUT = 4u;   // a bounded device-side wait gave up

constexpr int kGX = 32;  // stored column of node x = 0
constexpr int kGY = 2;   // stored row of node y = 0

// Geometry of one lattice of the batch. flags: kGeomMask (a wall mask) and
// kGeomOpenX (an x-slab of a lattice split across contexts: its x edges are
// not periodic; the pulls across them read the frame columns x = -2, -1 and
// nx, nx + 1, which the halo exchange fills).
constexpr int kGeomMask = 1;
constexpr int kGeomOpenX = 2;
struct Geom {
    int nx, ny, pitch, flags;
    long long f_off;     // element offset of plane 0 in the distribution arrays
    long long plane;     // elements per plane ((ny + 2 kGY) * pitch)
    long long mask_off;  // byte offset of this lattice's mask plane
    long long node_off;  // offset of this lattice in concatenated host arrays
};

__host__ __device__ __forceinline__ int node_index(const Geom& g, int x, int y) {
    return (y + kGY) * g.pitch + x + kGX;
}
__host__ __device__ __forceinline__ bool geom_mask(const Geom& g) { return (g.flags & kGeomMask) != 0; }
__host__ __device__ __forceinline__ bool geom_open_x(const Geom& g) { return (g.flags & kGeomOpenX) != 0; }

// Physical parameters of one lattice in the arithmetic type T.
template <typename T>
struct Phys {
    T rho_ref;            // deviation reference (0 for plain storage)
    T RT, a, b4;          // Eq. 15: R*T, a, b/4
    T G;                  // Eq. 7 / Eq. 13 interaction strength
    T kpsi;               // 2 / (G c^2) of Eq. 13
    T cs2;                // lattice sound speed squared, 1/3
    T s[9];               // diagonal of Lambda, Eq. 2
    T h[9];               // 1 - s/2, the factor of S in Eq. 3
    T li_e, li_z;         // s_e * 0.75 eps and s_zeta * 0.75 eps (Li's term after (1 - s/2))
    T b1;                 // b of the van der Waals and Peng-Robinson EOS
    T eps12, inv_eps12;   // eps of Eq. 12 and 1 / eps (0 when eps = 0)
    int eos;              // EOS_CS, EOS_VDW, EOS_PR (a holds a alpha(T)), PSI_EXP (Eq. 12)
};

constexpr int EOS_CS = 0;
constexpr int EOS_VDW = 1;
constexpr int EOS_PR = 2;
constexpr int PSI_EXP = 3;

// One CTA's piece of work: a tile of lattice `lat` with origin (x0, y0);
// clear = 1 when neither the tile nor its two-cell frame holds a solid cell
// (set by the host from the wall mask; always 1 without walls).
struct Tile {
    int lat, x0, y0, clear;
};

// A tile with a copy of its lattice's geometry, so that a CTA learns both
// with one round trip to memory (four independent 16-byte loads) instead of
// a tile load followed by a dependent geometry load.
struct alignas(16) TileGeom {
    Geom g;
    Tile t;
};

__device__ __forceinline__ int wrap_index(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Stored index of node (x, y) and the offsets from it to its four axis
// neighbours on the periodic lattice (Eq. 5 with periodic boundaries): the
// neighbour across an edge is the node at the far side of the same row or
// column. x in [-1, nx] and y in [-1, ny] (one period outside at most) are
// first brought into the lattice, so a halo cell beside an edge is the node
// it stands for. Valid for any nx, ny >= 1. With open_x (an x-slab) x is not
// wrapped: x = -1 and x = nx are the frame columns that hold the neighbouring
// slabs' edge columns, and their x neighbours the next frame columns.
struct Nbr {
    int c, xm, xp, ym, yp;
};
__device__ __forceinline__ Nbr nbr_of(int nx, int ny, int pitch, int x, int y, bool open_x = false) {
    if (!open_x) x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    Nbr n;
    n.c = (y + kGY) * pitch + x + kGX;
    n.xm = (x == 0 && !open_x) ? nx - 1 : -1;
    n.xp = (x == nx - 1 && !open_x) ? 1 - nx : 1;
    n.ym = y == 0 ? (ny - 1) * pitch : -pitch;
    n.yp = y == ny - 1 ? (1 - ny) * pitch : pitch;
    return n;
}
__device__ __forceinline__ Nbr nbr_geom(const Geom& g, int x, int y) {
    return nbr_of(g.nx, g.ny, g.pitch, x, y, geom_open_x(g));
}

// psi of Eq. 13 with the CS pressure of Eq. 15, written as
// psi^2 = kpsi * rho * (R T Z(eta) - a rho - c_s^2), Z = (1+h+h^2-h^3)/(1-h)^3.
// Near the density where psi^2 = 0 the bracket cancels; the FP32 version
// (vpsi below) recomputes it in FP64 there. psi^2 < 0 is clamped to 0 and
// flagged.
// The EOS helpers below spell every operation as an explicitly rounded
// intrinsic, so that no multiply-add is contracted differently in the
// kernels that inline them: every step kernel then computes bitwise the same
// psi.
__device__ __forceinline__ double psi_bracket_fp64(double rho, double RT, double a,
                                                   double b4, double cs2) {
    const double eta = __dmul_rn(b4, rho);
    const double om = __dsub_rn(1.0, eta);
    const double num = __dadd_rn(1.0, __dmul_rn(eta, __dadd_rn(1.0, __dmul_rn(eta, __dsub_rn(1.0, eta)))));
    const double z = __ddiv_rn(num, __dmul_rn(__dmul_rn(om, om), om));
    return __dsub_rn(__dsub_rn(__dmul_rn(RT, z), __dmul_rn(a, rho)), cs2);
}

// p / rho - c_s^2 of the van der Waals (d = 1) or Peng-Robinson EOS, with
// om = 1 - b rho (the pole at b rho = 1) and a the attraction (a alpha for PR).
__device__ __forceinline__ double bracket_cubic_fp64(double rho, double RT, double a, double b, double cs2,
                                                     bool pr) {
    const double br = __dmul_rn(b, rho);
    const double om = __dsub_rn(1.0, br);
    const double att = pr ? __ddiv_rn(__dmul_rn(a, rho), __dadd_rn(1.0, __dmul_rn(br, __dsub_rn(2.0, br))))
                          : __dmul_rn(a, rho);
    return __dsub_rn(__dsub_rn(__ddiv_rn(RT, om), att), cs2);
}

// psi of Eq. 12: exp(-1/rho) (eps = 0) or (rho / (eps + rho))^(1/eps).
__device__ __forceinline__ double psi_exp_fp64(double rho, double eps, double inv_eps) {
    return eps == 0.0 ? exp(__ddiv_rn(-1.0, rho)) : exp(__dmul_rn(log(__ddiv_rn(rho, __dadd_rn(eps, rho))), inv_eps));
}

__device__ __forceinline__ double psi_of(double rho, const Phys<double>& P, unsigned& flag) {
    if (P.eos == PSI_EXP) {
        if (!(rho > 0.0 && rho < 1.0e300)) {
            flag |= FLAG_NONFINITE;
            return 0.0;
        }
        return psi_exp_fp64(rho, P.eps12, P.inv_eps12);
    }
    const bool cubic = P.eos != EOS_CS;
    double q = cubic ? bracket_cubic_fp64(rho, P.RT, P.a, P.b1, P.cs2, P.eos == EOS_PR)
                     : psi_bracket_fp64(rho, P.RT, P.a, P.b4, P.cs2);
    double psi2 = __dmul_rn(__dmul_rn(P.kpsi, rho), q);
    const bool dense_ok = __dsub_rn(1.0, __dmul_rn(cubic ? P.b1 : P.b4, rho)) > 0.0;
    if (!(psi2 >= 0.0 && dense_ok)) {
        flag |= (psi2 < 0.0 && dense_ok) ? FLAG_PSI_CLAMPED : FLAG_NONFINITE;
        psi2 = 0.0;
    } else if (psi2 > 1.0e300) {
        flag |= FLAG_NONFINITE;
    }
    return sqrt(psi2);
}

__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Population and mask accesses of the step. Debug builds (-DLBM_DEBUG)
// check each index against the lattice's nine planes (one plane for the
// mask): an index outside reads NaN (a population) or solid (the mask) and a
// store outside is skipped, so a wrong offset shows up as a wrong or
// non-finite result in the parity tests instead of touching memory that
// belongs to another lattice. Release builds access directly.
template <typename T>
__device__ __forceinline__ T ld_pop(const T* __restrict__ p, int i, int n) {
#ifdef LBM_DEBUG
    if (i < 0 || i >= n) return T(NAN);
#endif
    return p[i];
}
// Populations are stored with the streaming hint (evict first): the step
// never reads what it writes, so L2 keeps the lines it reads, which
// neighbouring tiles read again for their halos (1-3% on batches larger than
// L2, no change on the bench batch).
template <typename T>
__device__ __forceinline__ void st_pop(T* __restrict__ p, int i, int n, T v) {
#ifdef LBM_DEBUG
    if (i < 0 || i >= n) return;
#endif
    __stcs(p + i, v);
}
__device__ __forceinline__ uint8_t ld_mask(const uint8_t* __restrict__ m, int i, int n) {
#ifdef LBM_DEBUG
    if (i < 0 || i >= n) return 1;
#endif
    return m[i];
}

// Opposite velocity: e_opp(a) = -e_a.
__host__ __device__ constexpr int opp(int a) {
    return a == 0 ? 0 : (a < 5 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5);
}

// Layouts of a stored state. Two-buffer storage (kLayoutPull) keeps the
// post-collision values of the last step, f*_a(x) in plane a at x, and the
// next step pulls them. In-place storage (one array, the AA pattern)
// alternates between two layouts:
//   kLayoutNatural  plane a at x holds f_a(x), already streamed;
//   kLayoutSwapped  plane opp(a) at x holds f*_a(x), streaming pending.
// A step from the natural layout collides every node in place and writes
// f*_a to plane opp(a) of the same node (swapped layout); a step from the
// swapped layout gathers f_a(x) from plane opp(a) at x - e_a (plane a at x
// when x - e_a is solid) and writes f*_a to plane a at x + e_a (plane
// opp(a) at x when x + e_a is solid), which is the natural layout again.
// Each node reads and writes only slots no other node touches in that step.
constexpr int kLayoutPull = 0;
constexpr int kLayoutNatural = 1;
constexpr int kLayoutSwapped = 2;

// Gather the distribution of node n after streaming (Eq. 5) from the
// post-collision array `fin` (pull form): f_a(x) = f*_a(x - e_a), with x - e_a
// taken periodically. With a wall mask, a link whose source is solid is
// reflected: f_a(x) = f*_abar(x). Returns true if the node itself is solid
// (then f is not filled). SWAP reads f*_a from plane opp(a) instead of
// plane a (the swapped layout of in-place storage).
template <typename T, bool SWAP = false>
__device__ __forceinline__ bool pull_node(const T* __restrict__ fin, const uint8_t* __restrict__ mask,
                                          int plane, const Nbr& n, T f[9]) {
    const int np = 9 * plane;  // < 2^31 (checked when the lattice is created)
    auto F = [&](int a, int i) { return ld_pop<T>(fin, (SWAP ? opp(a) : a) * plane + i, np); };
    const int c = n.c;
    if (mask != nullptr) {
        auto M = [&](int i) { return ld_mask(mask, i, plane); };
        if (M(c)) return true;
        f[0] = F(0, c);
        f[1] = M(c + n.xm)        ? F(3, c) : F(1, c + n.xm);
        f[2] = M(c + n.ym)        ? F(4, c) : F(2, c + n.ym);
        f[3] = M(c + n.xp)        ? F(1, c) : F(3, c + n.xp);
        f[4] = M(c + n.yp)        ? F(2, c) : F(4, c + n.yp);
        f[5] = M(c + n.ym + n.xm) ? F(7, c) : F(5, c + n.ym + n.xm);
        f[6] = M(c + n.ym + n.xp) ? F(8, c) : F(6, c + n.ym + n.xp);
        f[7] = M(c + n.yp + n.xp) ? F(5, c) : F(7, c + n.yp + n.xp);
        f[8] = M(c + n.yp + n.xm) ? F(6, c) : F(8, c + n.yp + n.xm);
        return false;
    }
    f[0] = F(0, c);
    f[1] = F(1, c + n.xm);
    f[2] = F(2, c + n.ym);
    f[3] = F(3, c + n.xp);
    f[4] = F(4, c + n.yp);
    f[5] = F(5, c + n.ym + n.xm);
    f[6] = F(6, c + n.ym + n.xp);
    f[7] = F(7, c + n.yp + n.xp);
    f[8] = F(8, c + n.yp + n.xm);
    return false;
}

// The distribution of node n in any layout (see kLayoutPull): the pull of
// two-buffer storage, the node's own planes (natural layout) or the pull
// from the opposite planes (swapped layout). Returns true if the node is
// solid.
template <typename T>
__device__ __forceinline__ bool gather_node(int layout, const T* __restrict__ f, const uint8_t* __restrict__ mask,
                                            int plane, const Nbr& n, T out[9]) {
    if (layout == kLayoutNatural) {
        if (mask != nullptr && ld_mask(mask, n.c, plane)) return true;
#pragma unroll
        for (int a = 0; a < 9; ++a) out[a] = ld_pop<T>(f, a * plane + n.c, 9 * plane);
        return false;
    }
    return layout == kLayoutSwapped ? pull_node<T, true>(f, mask, plane, n, out)
                                    : pull_node<T, false>(f, mask, plane, n, out);
}

// Offset from a node to its neighbour x + e_a (a = 1 .. 8) on the periodic
// lattice, from the node's Nbr.
__device__ __forceinline__ int nbr_offset(const Nbr& n, int a) {
    switch (a) {
        case 1: return n.xp;
        case 2: return n.yp;
        case 3: return n.xm;
        case 4: return n.ym;
        case 5: return n.yp + n.xp;
        case 6: return n.yp + n.xm;
        case 7: return n.ym + n.xm;
        default: return n.ym + n.xp;
    }
}

// The post-collision values f*_a of node n (the values the last step
// wrote for it) in any layout: plane a at the node (two-buffer storage),
// plane opp(a) at the node (swapped), or where streaming put them (natural:
// plane a at x + e_a, plane opp(a) at the node when x + e_a is solid).
template <typename T>
__device__ __forceinline__ void post_collision_node(int layout, const T* __restrict__ f,
                                                    const uint8_t* __restrict__ mask, int plane, const Nbr& n,
                                                    T out[9]) {
    const int np = 9 * plane;
    for (int a = 0; a < 9; ++a) {
        int slot = a, i = n.c;
        if (layout == kLayoutSwapped) {
            slot = opp(a);
        } else if (layout == kLayoutNatural && a > 0) {
            const int t = n.c + nbr_offset(n, a);
            if (mask != nullptr && ld_mask(mask, t, plane))
                slot = opp(a);
            else
                i = t;
        }
        out[a] = ld_pop<T>(f, slot * plane + i, np);
    }
}

// pull_node for a node at stored index c whose eight neighbours all lie
// inside the lattice (no wrap) and are fluid: fixed offsets only.
template <typename T>
__device__ __forceinline__ void pull_inner(const T* __restrict__ fin, int plane, int pitch, int c, T f[9]) {
    const int np = 9 * plane;
    auto F = [&](int a, int i) { return ld_pop<T>(fin, a * plane + i, np); };
    f[0] = F(0, c);
    f[1] = F(1, c - 1);
    f[2] = F(2, c - pitch);
    f[3] = F(3, c + 1);
    f[4] = F(4, c + pitch);
    f[5] = F(5, c - pitch - 1);
    f[6] = F(6, c - pitch + 1);
    f[7] = F(7, c + pitch + 1);
    f[8] = F(8, c + pitch - 1);
}

// Write the nine values of node (x, y), 0 <= x < nx, 0 <= y < ny; `base` is
// plane 0 of the lattice.
template <typename T>
__device__ __forceinline__ void store_node(T* __restrict__ base, const Geom& g, int x, int y,
                                           const T v[9]) {
    const int c = node_index(g, x, y);
    const int plane = (int)g.plane;
#pragma unroll
    for (int a = 0; a < 9; ++a) st_pop<T>(base, a * plane + c, 9 * plane, v[a]);
}

// Sum of the eight moving populations in a fixed association; the density
// is f_0 + sum8, and the collision sets f*_0 = drho - sum8(f*) with the same
// association.
template <typename T>
__device__ __forceinline__ T sum8(const T f[9]) {
    return ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
}

template <typename T>
__device__ __forceinline__ T sum9(const T f[9]) {
    return f[0] + sum8(f);
}

// Collision of one fluid node in moment space (Eq. 3) with m_eq of Eq. 4,
// the velocity of Eq. 6 and Li's source of Eq. 14, followed by f* = M^-1 m*.
// f holds the stored deviation f_a - w_a rho_ref on entry and the
// post-collision deviation on exit (M w = (1, -2, 1, 0, ...), so the constant
// part cancels in m - m_eq and M^-1 maps it back). drho = rho - rho_ref.
// (Fx, Fy) = -G psi (gx, gy) with g = sum_a w_a psi(x + e_a) e_a (Eq. 7);
// |F|^2 / psi^2 of Eq. 14 is G^2 |g|^2, and (1 - s/2) / (tau - 1/2) = s, so
// Li's terms enter m* as +s_e 0.75 eps G^2 |g|^2 and -s_zeta 0.75 eps G^2 |g|^2.
// For the momentum rows, m_eq = rho v = j + F/2 makes
// j - s_j (j - rho v) + (1 - s_j/2) F equal to j + F for every s_j.
template <typename T>
__device__ __forceinline__ void collide(T f[9], T rho, T drho, T Fx, T Fy, T g2G2,
                                        const Phys<T>& P) {
    const T half = T(0.5);
    // first moments and velocity, Eq. 6
    const T sx = f[1] - f[3];
    const T sy = f[2] - f[4];
    const T d57 = f[5] - f[7];
    const T d68 = f[6] - f[8];
    const T jx = sx + (d57 - d68);
    const T jy = sy + (d57 + d68);
    const T rvx = jx + half * Fx;       // rho v_x
    const T rvy = jy + half * Fy;
    const T inv_rho = recip(rho);
    const T vx = rvx * inv_rho;
    const T vy = rvy * inv_rho;

    // m = M f (deviation)
    const T p13 = f[1] + f[3], p24 = f[2] + f[4];
    const T p57 = f[5] + f[7], p68 = f[6] + f[8];
    const T a14 = p13 + p24;
    const T a58 = p57 + p68;
    const T m1 = T(2) * a58 - a14 - T(4) * f[0];
    const T m2 = T(4) * f[0] + a58 - T(2) * a14;
    const T m4 = (d57 - d68) - T(2) * sx;
    const T m6 = (d57 + d68) - T(2) * sy;
    const T m7 = p13 - p24;
    const T m8 = p57 - p68;

    // m_eq of Eq. 4 (deviation form: the rho_ref parts of rho, e, zeta cancel)
    const T ru2 = rvx * vx + rvy * vy;  // rho |v|^2
    const T meq1 = T(3) * ru2 - T(2) * drho;
    const T meq2 = drho - T(3) * ru2;
    const T meq7 = rvx * vx - rvy * vy;
    const T meq8 = rvx * vy;

    // source S of Eq. 14 (Eq. 8 plus Li's terms); m* = m - s (m - m_eq) + (1 - s/2) S
    const T vF6 = T(6) * (vx * Fx + vy * Fy);
    const T ms1 = m1 - P.s[1] * (m1 - meq1) + P.h[1] * vF6 + P.li_e * g2G2;
    const T ms2 = m2 - P.s[2] * (m2 - meq2) - P.h[2] * vF6 - P.li_z * g2G2;
    const T ms3 = jx + Fx;
    const T ms4 = m4 - P.s[4] * (m4 + rvx) - P.h[4] * Fx;
    const T ms5 = jy + Fy;
    const T ms6 = m6 - P.s[6] * (m6 + rvy) - P.h[6] * Fy;
    const T ms7 = m7 - P.s[7] * (m7 - meq7) + P.h[7] * (T(2) * (vx * Fx - vy * Fy));
    const T ms8 = m8 - P.s[8] * (m8 - meq8) + P.h[8] * (vx * Fy + vy * Fx);

    // f* = M^-1 m* = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) m*
    const T a0 = drho * T(1.0 / 9.0);
    const T a1 = ms1 * T(1.0 / 36.0);
    const T a2 = ms2 * T(1.0 / 36.0);
    const T a3 = ms3 * T(1.0 / 6.0);
    const T a4 = ms4 * T(1.0 / 12.0);
    const T a5 = ms5 * T(1.0 / 6.0);
    const T a6 = ms6 * T(1.0 / 12.0);
    const T a7 = ms7 * T(0.25);
    const T a8 = ms8 * T(0.25);
    const T axis = a0 - a1 - T(2) * a2;
    const T diag = a0 + T(2) * a1 + a2;
    const T px = a3 - T(2) * a4;
    const T py = a5 - T(2) * a6;
    const T qx = a3 + a4;
    const T qy = a5 + a6;
    f[1] = axis + px + a7;
    f[2] = axis + py - a7;
    f[3] = axis - px + a7;
    f[4] = axis - py - a7;
    f[5] = diag + qx + qy + a8;
    f[6] = diag - qx + qy - a8;
    f[7] = diag - qx - qy + a8;
    f[8] = diag + qx - qy - a8;
    // f*_0 = a0 - 4 a1 + 4 a2 in exact arithmetic. Taking it as the remainder
    // drho - sum8(f*) instead makes the next step's density f*_0 + sum8(f*)
    // return drho exactly wherever the subtraction is exact (sum8 within a
    // factor 2 of drho, as in any phase near rest). Otherwise the rounded 1/9
    // and the identical rounding of every node of a uniform phase would shift
    // the mass by the same relative amount at every step.
    f[0] = drho - sum8(f);
}

// ---------------------------------------------------------------------------
// FP32 arithmetic in explicit IEEE operations, one node (F1) or two nodes per
// paired instruction (F2: FADD2 / FMUL2 / FFMA2 on sm_100+). Every operation
// is the same correctly rounded operation in both forms and nothing is left
// for the compiler to contract, so one node gives bitwise the same result
// whether it is computed alone or paired with another.
struct F1 {
    float v;
};
struct F2 {
    float2 v;
};
__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return {__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return {__fsub_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return {__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 vfma(F1 a, F1 b, F1 c) { return {__fmaf_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
// a - b as fma(b, -1, a): the product is exact, so this is round(a - b)
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }

template <class V> __device__ __forceinline__ V splat(float s);
template <> __device__ __forceinline__ F1 splat<F1>(float s) { return {s}; }
template <> __device__ __forceinline__ F2 splat<F2>(float s) { return {make_float2(s, s)}; }

// per-lane helpers: quotient, reciprocal square root, lane access
__device__ __forceinline__ F1 vdiv(F1 a, F1 b) { return {__fdividef(a.v, b.v)}; }
__device__ __forceinline__ F2 vdiv(F2 a, F2 b) {
    return {make_float2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y))};
}
__device__ __forceinline__ int lanes(F1) { return 1; }
__device__ __forceinline__ int lanes(F2) { return 2; }
__device__ __forceinline__ float lane(F1 a, int) { return a.v; }
__device__ __forceinline__ float lane(F2 a, int i) { return i == 0 ? a.v.x : a.v.y; }
__device__ __forceinline__ void set_lane(F1& a, int, float x) { a.v = x; }
__device__ __forceinline__ void set_lane(F2& a, int i, float x) {
    if (i == 0) a.v.x = x; else a.v.y = x;
}

// Density sum of the FP32 path: f_0 plus the eight moving populations in
// the association ((f1 + f3) + (f2 + f4)) + ((f5 + f7) + (f6 + f8)), whose
// partial sums are also the pair sums of m = M f (vcollide).
template <class V>
__device__ __forceinline__ V vsum8(const V f[9]) {
    return ((f[1] + f[3]) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
}
template <class V>
__device__ __forceinline__ V vsum9(const V f[9]) {
    return f[0] + vsum8(f);
}

// Square root by the hardware approximation (sqrt.approx, relative error
// about 2^-23; subnormal inputs flush to zero).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// psi of Eq. 13 (see psi_of above): the polynomial in explicit operations, the
// quotient per lane with the fast hardware approximation, the FP64 fallback
// near the psi = 0 root, and per lane one combined test of the three
// conditions that need a flag (psi^2 < 0, non-finite, eta >= 1), whose rare
// failure is sorted out off the common path.
template <class V>
__device__ __forceinline__ V vpsi(V rho, const Phys<float>& P, unsigned& flag) {
    const V one = splat<V>(1.0f);
    const V eta = splat<V>(P.b4) * rho;
    const V om = one - eta;
    const V num = vfma(eta, vfma(eta, one - eta, one), one);
    const V C = vdiv(num, (om * om) * om);
    V q = vfma(splat<V>(P.RT), C, splat<V>(0.0f) - vfma(splat<V>(P.a), rho, splat<V>(P.cs2)));
    V psi2 = (splat<V>(P.kpsi) * rho) * q;
    V out;
#pragma unroll
    for (int i = 0; i < lanes(V{}); ++i) {
        float p2 = lane(psi2, i);
        const float qi = lane(q, i), ri = lane(rho, i), omi = lane(om, i);
        if (fabsf(qi) < 0.0078125f * P.cs2)
            p2 = __fmul_rn(__fmul_rn(P.kpsi, ri),
                           (float)psi_bracket_fp64((double)ri, (double)P.RT, (double)P.a, (double)P.b4,
                                                   (double)P.cs2));
        if (!(p2 >= 0.0f && p2 <= 3.0e38f && omi > 0.0f)) {
            flag |= (p2 < 0.0f && omi > 0.0f) ? FLAG_PSI_CLAMPED : FLAG_NONFINITE;
            p2 = 0.0f;
        }
        set_lane(out, i, sqrt_approx(p2));
    }
    return out;
}

// psi for the EOS other than Carnahan-Starling, one lane at a time (general
// path only): van der Waals and Peng-Robinson through Eq. 13 with the same
// FP64 fallback near the psi = 0 root and the same flags as vpsi, Eq. 12 by
// expf/logf.
__device__ __forceinline__ float psi_variant(float rho, const Phys<float>& P, unsigned& flag) {
    if (P.eos == PSI_EXP) {
        if (!(rho > 0.0f && rho <= 3.0e38f)) {
            flag |= FLAG_NONFINITE;
            return 0.0f;
        }
        return P.eps12 == 0.0f ? expf(__fdiv_rn(-1.0f, rho))
                               : expf(__fmul_rn(logf(__fdiv_rn(rho, __fadd_rn(P.eps12, rho))), P.inv_eps12));
    }
    const bool pr = P.eos == EOS_PR;
    const float br = __fmul_rn(P.b1, rho);
    const float om = __fsub_rn(1.0f, br);
    const float att = pr ? __fdiv_rn(__fmul_rn(P.a, rho), __fmaf_rn(br, __fsub_rn(2.0f, br), 1.0f))
                         : __fmul_rn(P.a, rho);
    const float q = __fsub_rn(__fsub_rn(__fdiv_rn(P.RT, om), att), P.cs2);
    float p2 = __fmul_rn(__fmul_rn(P.kpsi, rho), q);
    if (fabsf(q) < 0.0078125f * P.cs2)
        p2 = (float)__dmul_rn(__dmul_rn((double)P.kpsi, (double)rho),
                              bracket_cubic_fp64((double)rho, (double)P.RT, (double)P.a, (double)P.b1,
                                                 (double)P.cs2, pr));
    if (!(p2 >= 0.0f && p2 <= 3.0e38f && om > 0.0f)) {
        flag |= (p2 < 0.0f && om > 0.0f) ? FLAG_PSI_CLAMPED : FLAG_NONFINITE;
        p2 = 0.0f;
    }
    return sqrt_approx(p2);
}

// psi of any kind: the paired Carnahan-Starling form, else lane by lane.
template <class V>
__device__ __forceinline__ V vpsi_any(V rho, const Phys<float>& P, unsigned& flag) {
    if (P.eos == EOS_CS) return vpsi(rho, P, flag);
    V out;
#pragma unroll
    for (int i = 0; i < lanes(V{}); ++i) set_lane(out, i, psi_variant(lane(rho, i), P, flag));
    return out;
}

// Force sum of Eq. 7 (see force_sum below) in explicit operations.
template <class V>
__device__ __forceinline__ void vforce_sum(V pe, V pn, V pw, V ps, V pne, V pnw, V psw, V pse, V& gx, V& gy) {
    const V third = splat<V>(1.0f / 3.0f), twelfth = splat<V>(1.0f / 12.0f);
    gx = vfma(third, pe - pw, twelfth * ((pne - pnw) + (pse - psw)));
    gy = vfma(third, pn - ps, twelfth * ((pne + pnw) - (psw + pse)));
}

// The collision of collide<T> (same equations, same order of terms) in
// explicit operations, for one node (F1) or a pair of nodes (F2).
template <class V>
__device__ __forceinline__ void vcollide(V f[9], V rho, V drho, V Fx, V Fy, V g2G2, const Phys<float>& P) {
    const V half = splat<V>(0.5f), two = splat<V>(2.0f), three = splat<V>(3.0f), four = splat<V>(4.0f);
    const V sx = f[1] - f[3];
    const V sy = f[2] - f[4];
    const V d57 = f[5] - f[7];
    const V d68 = f[6] - f[8];
    const V jx = sx + (d57 - d68);
    const V jy = sy + (d57 + d68);
    const V rvx = vfma(half, Fx, jx);
    const V rvy = vfma(half, Fy, jy);
    const V inv_rho = vdiv(splat<V>(1.0f), rho);
    const V vx = rvx * inv_rho;
    const V vy = rvy * inv_rho;

    const V p13 = f[1] + f[3], p24 = f[2] + f[4];
    const V p57 = f[5] + f[7], p68 = f[6] + f[8];
    const V a14 = p13 + p24;
    const V a58 = p57 + p68;
    const V f0 = f[0];
    const V m1 = vfma(two, a58, splat<V>(0.0f) - vfma(four, f0, a14));
    const V m2 = vfma(four, f0, a58) - two * a14;
    const V m4 = (d57 - d68) - two * sx;
    const V m6 = (d57 + d68) - two * sy;
    const V m7 = p13 - p24;
    const V m8 = p57 - p68;

    const V ru2 = vfma(rvx, vx, rvy * vy);
    const V meq1 = vfma(three, ru2, splat<V>(0.0f) - two * drho);
    const V meq2 = drho - three * ru2;
    const V meq7 = vfma(rvx, vx, splat<V>(0.0f) - rvy * vy);
    const V meq8 = rvx * vy;

    const V vF6 = splat<V>(6.0f) * vfma(vx, Fx, vy * Fy);
    // m* = m - s (m - m_eq) + (1 - s/2) S, then scaled by 1 / |row|^2 of M
    const V ms1 = vfma(splat<V>(P.li_e), g2G2, vfma(splat<V>(P.h[1]), vF6, m1 - splat<V>(P.s[1]) * (m1 - meq1)));
    const V ms2 = vfma(splat<V>(-P.li_z), g2G2, m2 - splat<V>(P.s[2]) * (m2 - meq2) - splat<V>(P.h[2]) * vF6);
    const V ms3 = jx + Fx;
    const V ms4 = (m4 - splat<V>(P.s[4]) * (m4 + rvx)) - splat<V>(P.h[4]) * Fx;
    const V ms5 = jy + Fy;
    const V ms6 = (m6 - splat<V>(P.s[6]) * (m6 + rvy)) - splat<V>(P.h[6]) * Fy;
    const V S7 = two * vfma(vx, Fx, splat<V>(0.0f) - vy * Fy);
    const V S8 = vfma(vx, Fy, vy * Fx);
    const V ms7 = vfma(splat<V>(P.h[7]), S7, m7 - splat<V>(P.s[7]) * (m7 - meq7));
    const V ms8 = vfma(splat<V>(P.h[8]), S8, m8 - splat<V>(P.s[8]) * (m8 - meq8));

    const V a0 = drho * splat<V>(1.0f / 9.0f);
    const V a1 = ms1 * splat<V>(1.0f / 36.0f);
    const V a2 = ms2 * splat<V>(1.0f / 36.0f);
    const V a3 = ms3 * splat<V>(1.0f / 6.0f);
    const V a4 = ms4 * splat<V>(1.0f / 12.0f);
    const V a5 = ms5 * splat<V>(1.0f / 6.0f);
    const V a6 = ms6 * splat<V>(1.0f / 12.0f);
    const V a7 = ms7 * splat<V>(0.25f);
    const V a8 = ms8 * splat<V>(0.25f);
    const V axis = (a0 - a1) - two * a2;
    const V diag = vfma(two, a1, a0) + a2;
    const V px = a3 - two * a4;
    const V py = a5 - two * a6;
    const V qx = a3 + a4;
    const V qy = a5 + a6;
    f[1] = (axis + px) + a7;
    f[2] = (axis + py) - a7;
    f[3] = (axis - px) + a7;
    f[4] = (axis - py) - a7;
    f[5] = ((diag + qx) + qy) + a8;
    f[6] = ((diag - qx) + qy) - a8;
    f[7] = ((diag - qx) - qy) + a8;
    f[8] = ((diag + qx) - qy) - a8;
    // f*_0: the rest population takes the difference between the moving
    // populations the node received and those it sends on,
    //   f*_0 = f_0 + (a14 - b14) + (a58 - b58),
    // which in exact arithmetic is drho - sum_{a>=1} f*_a (collide). Near
    // rest the two differences are exact (Sterbenz) and small, so the only
    // rounding of the node's mass is that of the last addition, instead of
    // the roundings of the two eight-term sums in drho - sum8(f*). In a
    // steady field (a bulk phase, a flat interface) each step repeats the
    // same roundings, so those made the mass drift linearly (2e-6 over 2000
    // steps of the slab batch; 2e-8 in this form).
    const V b14 = (f[1] + f[3]) + (f[2] + f[4]);
    const V b58 = (f[5] + f[7]) + (f[6] + f[8]);
    f[0] = f0 + ((a14 - b14) + (a58 - b58));
}

// Force sum g = sum_a w_a psi(x + e_a) e_a of Eq. 7 from the nine psi values
// of a 3x3 neighbourhood; on lattices with walls a negative entry marks a
// solid neighbour, which takes the centre node's psi.
template <typename T>
__device__ __forceinline__ void force_sum(bool walls, T c, T pe, T pn, T pw, T ps, T pne, T pnw,
                                          T psw, T pse, T& gx, T& gy) {
    if (walls) {
        pe = pe < T(0) ? c : pe;
        pn = pn < T(0) ? c : pn;
        pw = pw < T(0) ? c : pw;
        ps = ps < T(0) ? c : ps;
        pne = pne < T(0) ? c : pne;
        pnw = pnw < T(0) ? c : pnw;
        psw = psw < T(0) ? c : psw;
        pse = pse < T(0) ? c : pse;
    }
    const T third = T(1.0 / 3.0), twelfth = T(1.0 / 12.0);
    gx = third * (pe - pw) + twelfth * ((pne - pnw) + (pse - psw));
    gy = third * (pn - ps) + twelfth * ((pne + pnw) - (psw + pse));
}

}  // namespace lbm
