// Particle kernels (§2 of Günther et al., arXiv:1109.3277): moving
// bounce-back correction and momentum exchange (Eq. 4-5), anisotropic
// Hertz / Berne–Pechukas and lubrication pair forces (Eq. 6-9), the
// Newton–Euler update, and the node coverage with fill and empty.
//
// Per-particle work runs one CTA per particle over the particle's bounding
// box; per-particle sums are FP64 and reduced in a fixed order, so results
// are bit-reproducible run to run.
#include "lbe_internal.cuh"

namespace lbe {

namespace {

constexpr int PT = 128;  // threads per per-particle CTA

// ---------------------------------------------------------- geometry (FP64)
// The inside test is written with explicit round-to-nearest intrinsics so
// that no multiply-add is contracted: the quadric is evaluated in a fixed
// operation order.

__device__ __forceinline__ double m_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double a_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double s_(double a, double b) { return __dsub_rn(a, b); }

__device__ void rotmat(const double *q, double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = s_(1.0, m_(2.0, a_(m_(y, y), m_(z, z))));
    R[0][1] = m_(2.0, s_(m_(x, y), m_(w, z)));
    R[0][2] = m_(2.0, a_(m_(x, z), m_(w, y)));
    R[1][0] = m_(2.0, a_(m_(x, y), m_(w, z)));
    R[1][1] = s_(1.0, m_(2.0, a_(m_(x, x), m_(z, z))));
    R[1][2] = m_(2.0, s_(m_(y, z), m_(w, x)));
    R[2][0] = m_(2.0, s_(m_(x, z), m_(w, y)));
    R[2][1] = m_(2.0, a_(m_(y, z), m_(w, x)));
    R[2][2] = s_(1.0, m_(2.0, a_(m_(x, x), m_(y, y))));
}

__device__ __forceinline__ bool periodic_dim(const Lat &L, int k) { return k < 2 || !L.walls; }
__device__ __forceinline__ int ext_of(const Lat &L, int k) { return k == 0 ? L.nx : (k == 1 ? L.ny : L.nz); }

// Displacement of node coordinate xi from particle coordinate X: nearest
// periodic image, shifting the integer first and subtracting once.
__device__ __forceinline__ double node_disp(const Lat &L, int k, int xi, double X)
{
    if (periodic_dim(L, k)) {
        int n = ext_of(L, k);
        double s = rint(__ddiv_rn(s_((double)xi, X), (double)n));
        return s_((double)((long long)xi - (long long)s * n), X);
    }
    return s_((double)xi, X);
}

__device__ __forceinline__ double pair_disp(const Lat &L, int k, double a, double b)
{
    double r = s_(b, a);
    if (periodic_dim(L, k)) {
        double n = (double)ext_of(L, k);
        r = s_(r, m_(n, rint(__ddiv_rn(r, n))));
    }
    return r;
}

struct Geo {
    double R[3][3];
    float R32[3][3];
    double ip2, io2;
    float ip2f, io2f;
};

__device__ void geo_of(const double *q, double rp, double ro, Geo &g)
{
    rotmat(q, g.R);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) g.R32[a][b] = (float)g.R[a][b];
    g.ip2 = __ddiv_rn(1.0, m_(rp, rp));
    g.io2 = __ddiv_rn(1.0, m_(ro, ro));
    g.ip2f = (float)g.ip2;
    g.io2f = (float)g.io2;
}

// Inside test: an FP32 evaluation decides unless it lies within 1e-3 of the
// surface, where the exact FP64 evaluation (oracle operation order) decides.
// d32 is the displacement in FP32 (error ~1e-7 lattice units); dx the exact
// FP64 displacement, formed only when needed.
__device__ __forceinline__ bool inside_q32(const Geo &g, const float d[3], float &q32)
{
    float e[3];
#pragma unroll
    for (int k = 0; k < 3; k++) e[k] = g.R32[0][k] * d[0] + g.R32[1][k] * d[1] + g.R32[2][k] * d[2];
    q32 = e[0] * e[0] * g.ip2f + (e[1] * e[1] + e[2] * e[2]) * g.io2f;
    return q32 < 0.999f;
}

__device__ __forceinline__ bool inside_exact(const Geo &g, const double dx[3])
{
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        d[k] = a_(a_(m_(g.R[0][k], dx[0]), m_(g.R[1][k], dx[1])), m_(g.R[2][k], dx[2]));
    double qv = a_(a_(m_(m_(d[0], d[0]), g.ip2), m_(m_(d[1], d[1]), g.io2)), m_(m_(d[2], d[2]), g.io2));
    return qv <= 1.0;
}

struct Box {
    int lo[3], ext[3];  // lower corner in unwrapped coordinates, extents
    int full[3];        // the axis spans a whole period (nearest image taken per node)
    int count;
};

// Axis-aligned box containing the ellipsoid at X (not necessarily wrapped),
// widened by one node, as doubles: lo[k] = floor(X - h) - 1, hi[k] =
// ceil(X + h) + 1 with h the half-extent of the rotated ellipsoid along k.
// Non-finite geometry, or a centre further than 1e9 from the origin (a
// particle that has left any lattice), gives lo > hi: an empty box.
__device__ void box_of(const Lat &L, const double *X, const double R[3][3], double rp, double ro,
                       double lo[3], double hi[3])
{
    for (int k = 0; k < 3; k++) {
        double h = sqrt(rp * rp * R[k][0] * R[k][0] + ro * ro * (R[k][1] * R[k][1] + R[k][2] * R[k][2]));
        lo[k] = floor(X[k] - h) - 1.0;
        hi[k] = ceil(X[k] + h) + 1.0;
        if (!(lo[k] <= hi[k]) || !(fabs(X[k]) < 1e9) || !(h < 1e9)) {
            lo[k] = 1.0;
            hi[k] = 0.0;
        }
    }
}

__device__ __forceinline__ bool box_empty(const double lo[3], const double hi[3])
{
    return !(lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2]);
}

// Integer box over lattice nodes: along walls clamped to [0, n-1]; along
// periodic axes at most one period.  Coordinates stay unwrapped (relative to
// the particle, as the box was formed around it), so a node's displacement
// from the particle is one exact subtraction; an axis clamped to a whole
// period is flagged and takes the nearest image per node instead.  All
// arithmetic before the conversion to int is in double and |lo|, |hi| are
// below ~1e9 (box_of), so no int overflows.
__device__ void finish_box(const Lat &L, const double *lo_in, const double *hi_in, Box &b)
{
    bool empty = box_empty(lo_in, hi_in);
    for (int k = 0; k < 3; k++) {
        double n = (double)ext_of(L, k);
        double lo = lo_in[k], hi = hi_in[k];
        b.full[k] = 0;
        if (empty) {
            lo = 0.0;
            hi = -1.0;
        } else if (!periodic_dim(L, k)) {
            lo = fmax(lo, 0.0);
            hi = fmin(hi, n - 1.0);
        } else if (hi - lo + 1.0 > n) {
            lo = 0.0;
            hi = n - 1.0;
            b.full[k] = 1;
        }
        b.lo[k] = hi >= lo ? (int)lo : 0;
        b.ext[k] = hi >= lo ? (int)(hi - lo + 1.0) : 0;
    }
    b.count = b.ext[0] * b.ext[1] * b.ext[2];
}

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Box entry k: unwrapped coordinates u[3] and the wrapped node (x, y, z).
__device__ __forceinline__ void box_node(const Lat &L, const Box &b, int k, int u[3], int &x, int &y,
                                         int &z)
{
    int bx = k % b.ext[0];
    int t = k / b.ext[0];
    int by = t % b.ext[1];
    int bz = t / b.ext[1];
    u[0] = b.lo[0] + bx;
    u[1] = b.lo[1] + by;
    u[2] = b.lo[2] + bz;
    x = wrapi(u[0], L.nx);
    y = wrapi(u[1], L.ny);
    z = wrapi(u[2], L.nz);
}

// Displacement of a box node from the particle centre X (the centre the box
// was formed around), equal to the nearest-image displacement.
__device__ __forceinline__ double box_disp(const Lat &L, const Box &b, int k, int u, int w, double X)
{
    return b.full[k] ? node_disp(L, k, w, X) : s_((double)u, X);
}

__device__ __forceinline__ bool is_wall_z(const Lat &L, int z) { return L.walls && (z == 0 || z == L.nz - 1); }

// ---- candidate rows -------------------------------------------------------
// Along a row of the box (fixed unwrapped y, z) the nodes the inside test
// can accept lie in one x interval: where the quadric of the ellipsoid is
// at most 1.  The interval of the quadric at most QSPAN, widened by a node
// on each side, holds all of them whatever the FP32 rounding of its
// computation (relative errors ~1e-6 against a margin of ~1% of the radii),
// so only those candidates are tested.  Boxes that span a whole period use
// the plain box loop.
constexpr float QSPAN = 1.02f;

// x interval [xa, xb] (unwrapped, clamped to the box) of row (u1, u2) for
// the ellipsoid g at X; xa > xb when the row misses it.
__device__ __forceinline__ void row_span(const Geo &g, const double X[3], const Box &b, int u1, int u2, int &xa,
                                         int &xb)
{
    const float dy = (float)((double)u1 - X[1]), dz = (float)((double)u2 - X[2]);
    const float w[3] = {g.ip2f, g.io2f, g.io2f};
    float A = 0.f, B = 0.f, C = -QSPAN;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float r0 = g.R32[0][k], ck = __fmaf_rn(g.R32[1][k], dy, __fmul_rn(g.R32[2][k], dz));
        A = __fmaf_rn(w[k] * r0, r0, A);
        B = __fmaf_rn(2.f * w[k] * r0, ck, B);
        C = __fmaf_rn(w[k] * ck, ck, C);
    }
    const float D = __fmaf_rn(B, B, -4.f * A * C);
    xa = 1;
    xb = 0;
    if (!(D >= 0.f) || !(A > 0.f)) return;
    const float sq = sqrtf(D), ia = 0.5f / A;
    const double lo = X[0] + (double)((-B - sq) * ia), hi = X[0] + (double)((-B + sq) * ia);
    if (!(lo >= -2e9 && hi <= 2e9)) return;
    xa = max((int)floor(lo) - 1, b.lo[0]);
    xb = min((int)ceil(hi) + 1, b.lo[0] + b.ext[0] - 1);
}

__device__ __forceinline__ bool box_full(const Box &b) { return b.full[0] || b.full[1] || b.full[2]; }

// Every candidate node of a particle's box, each visited once.  Each warp
// takes chunks of 32 rows: lane l computes the NSEG disjoint segments
// [xs[j], xe[j]] of row l of the chunk (spans(u1, u2, xs, xe), empty when
// xs > xe, clamped to the box); a warp prefix over the rows' candidate
// counts flattens them, and the lanes take consecutive candidates.  No
// barrier: the warps of a CTA work on their own rows.  node(ux, u1, u2,
// valid) is called by all 32 lanes of a warp in whole passes (valid =
// false past the end), so it may use warp votes.  A box that spans a whole
// period visits all its nodes.
template <int NSEG, class SP, class F>
__device__ __forceinline__ void for_segments(const Box &b, SP spans, F node)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (box_full(b)) {
        for (int k0 = warp * 32; k0 < b.count; k0 += nw * 32) {
            const int k = k0 + lane;
            const bool valid = k < b.count;
            const int kk = valid ? k : 0;
            const int t = kk / b.ext[0];
            node(b.lo[0] + kk % b.ext[0], b.lo[1] + t % b.ext[1], b.lo[2] + t / b.ext[1], valid);
        }
        return;
    }
    const int rows = b.ext[1] * b.ext[2];
    for (int r0 = warp * 32; r0 < rows; r0 += nw * 32) {
        const int r = r0 + lane;
        int xs[NSEG], len[NSEG];
        int tot = 0;
        if (r < rows) {
            int xe[NSEG];
            spans(b.lo[1] + r % b.ext[1], b.lo[2] + r / b.ext[1], xs, xe);
#pragma unroll
            for (int j = 0; j < NSEG; j++) {
                len[j] = max(0, xe[j] - xs[j] + 1);
                tot += len[j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < NSEG; j++) {
                xs[j] = 0;
                len[j] = 0;
            }
        }
        int incl = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(full, incl, off);
            if (lane >= off) incl += v;
        }
        const int excl = incl - tot;
        const int total = __shfl_sync(full, incl, 31);
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < total;
            // the row (lane) holding candidate k: last lane with excl <= k
            int src = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int e = __shfl_sync(full, excl, src + step);
                if (e <= k) src += step;
            }
            int rem = k - __shfl_sync(full, excl, src);
            int ux = 0;
            bool found = false;
#pragma unroll
            for (int j = 0; j < NSEG; j++) {
                const int xj = __shfl_sync(full, xs[j], src), lj = __shfl_sync(full, len[j], src);
                if (!found && rem < lj) {
                    ux = xj + rem;
                    found = true;
                } else if (!found) {
                    rem -= lj;
                }
            }
            const int rr = r0 + src;
            node(ux, b.lo[1] + rr % b.ext[1], b.lo[2] + rr / b.ext[1], valid);
        }
    }
}

// The candidates of one ellipsoid (g at X) in box b.
template <class F>
__device__ __forceinline__ void for_candidates(const Box &b, const Geo &g, const double X[3], F node)
{
    for_segments<1>(b, [&](int u1, int u2, int *xs, int *xe) { row_span(g, X, b, u1, u2, xs[0], xe[0]); }, node);
}

// ---- coverage geometry ----------------------------------------------------
// The geometry the coverage kernels need of a particle, computed once per
// step by one thread per particle (k_geom) instead of by every CTA: the
// rotation and inverse squared radii, the centre the box was formed around
// with its integer and FP32 parts, and the box.
struct PGeom {
    Geo g;
    double X[3];
    int Xi[3];
    float Xf[3];
    Box box;
};

// Old geometry (the last coverage update's) and new geometry, and for the
// transition the new centre unwrapped next to the old one and the union of
// the two boxes.
struct PGeom2 {
    PGeom old_, now;
    double Xu[3];
    Box uni;
};

__device__ void pgeom_of(const Lat &L, const double *X, const double *q, double rp, double ro, PGeom &o)
{
    geo_of(q, rp, ro, o.g);
    double lo[3], hi[3];
    box_of(L, X, o.g.R, rp, ro, lo, hi);
    finish_box(L, lo, hi, o.box);
    for (int k = 0; k < 3; k++) {
        o.X[k] = X[k];
        // X = Xi + Xf, Xi integral: the FP32 displacement (u - Xi) - Xf
        // carries no large cancellation (box_of bounds |X| < 1e9)
        const double fl = floor(X[k]);
        o.Xi[k] = o.box.count ? (int)fl : 0;
        o.Xf[k] = (float)(X[k] - fl);
    }
}

__device__ __forceinline__ void geom_body(const Lat &L, const Parts &P, int p)
{
    PGeom2 &G = reinterpret_cast<PGeom2 *>(P.geo)[p];
    pgeom_of(L, P.Xold + 3 * p, P.qold + 4 * p, P.rp[p], P.ro[p], G.old_);
    pgeom_of(L, P.X + 3 * p, P.q + 4 * p, P.rp[p], P.ro[p], G.now);
    double lo[3], hi[3], lo2[3], hi2[3];
    for (int k = 0; k < 3; k++) G.Xu[k] = P.Xold[3 * p + k] + pair_disp(L, k, P.Xold[3 * p + k], P.X[3 * p + k]);
    box_of(L, P.Xold + 3 * p, G.old_.g.R, P.rp[p], P.ro[p], lo, hi);
    box_of(L, G.Xu, G.now.g.R, P.rp[p], P.ro[p], lo2, hi2);
    if (box_empty(lo, hi)) {
        for (int k = 0; k < 3; k++) {
            lo[k] = lo2[k];
            hi[k] = hi2[k];
        }
    } else if (!box_empty(lo2, hi2)) {
        for (int k = 0; k < 3; k++) {
            lo[k] = fmin(lo[k], lo2[k]);
            hi[k] = fmax(hi[k], hi2[k]);
        }
    }
    finish_box(L, lo, hi, G.uni);
}

__global__ void k_geom(Lat L, Parts P)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P.n) geom_body(L, P, p);
}

// Fixed-order block reduction of K doubles (PT threads).
template <int K>
__device__ void block_sum(double (&v)[K], double (*sh)[PT / 32])
{
#pragma unroll
    for (int k = 0; k < K; k++) {
        double a = v[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double a = 0.0;
            for (int w = 0; w < PT / 32; w++) a += sh[k][w];
            v[k] = a;
        }
    }
}

__device__ __forceinline__ int nbr_node(const Lat &L, int x, int y, int z, int i)
{
    int xx = x + cx(i), yy = y + cy(i), zz = z + cz(i);
    xx = xx < 0 ? xx + L.nx : (xx >= L.nx ? xx - L.nx : xx);
    yy = yy < 0 ? yy + L.ny : (yy >= L.ny ? yy - L.ny : yy);
    if (L.walls) {
        if (zz < 0 || zz >= L.nz) return -1;
    } else {
        zz = zz < 0 ? zz + L.nz : (zz >= L.nz ? zz - L.nz : zz);
    }
    return xx + L.nx * (yy + L.ny * zz);
}

// ------------------------------------------------------------ links
// For every link between a solid node x of particle p and a fluid node
// y = x + c_i: the population leaving y towards x was reflected into slot i
// of y by the streaming kernel (f*_ī(y)); add C = 6 w_i ρ^c(y) u_surf·c_i
// with u_surf = V + ω × r_b at the link midpoint (Eq. 4), and give the
// particle F = (2 f*_ī + C) c_ī and r_b × F (Eq. 5).

template <class S>
__global__ void __launch_bounds__(PT) k_links(Lat L, Parts P, typename S::P *__restrict__ fnew,
                                              const float *__restrict__ rho,
                                              const uint8_t *__restrict__ type,
                                              const uint32_t *__restrict__ owner)
{
    const int p = blockIdx.x;
    __shared__ Box box;
    __shared__ double sX[3];
    __shared__ float sV[3], sW[3];
    __shared__ double red[6][PT / 32];
    if (threadIdx.x == 0) {
        double R[3][3];
        rotmat(P.q + 4 * p, R);
        double lo[3], hi[3];
        box_of(L, P.X + 3 * p, R, P.rp[p], P.ro[p], lo, hi);
        finish_box(L, lo, hi, box);
        for (int k = 0; k < 3; k++) {
            sX[k] = P.X[3 * p + k];
            sV[k] = (float)P.V[3 * p + k];
            sW[k] = (float)P.W[3 * p + k];
        }
    }
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < box.count; k += PT) {
        int x, y, z, u[3];
        box_node(L, box, k, u, x, y, z);
        int n = x + L.nx * (y + L.ny * z);
        if (!idx_ok(L, n, L.N, 2)) continue;
        if (owner[n] != (uint32_t)p) continue;
        float dn[3] = {(float)box_disp(L, box, 0, u[0], x, sX[0]), (float)box_disp(L, box, 1, u[1], y, sX[1]),
                       (float)box_disp(L, box, 2, u[2], z, sX[2])};
        float aF[3] = {0.f, 0.f, 0.f}, aT[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 1; i < Q; i++) {
            int m = nbr_node(L, x, y, z, i);
            if (m < 0 || !idx_ok(L, m, L.N, 3) || type[m] != FLUID) continue;
            float rb[3] = {dn[0] + 0.5f * cx(i), dn[1] + 0.5f * cy(i), dn[2] + 0.5f * cz(i)};
            float us[3] = {sV[0] + sW[1] * rb[2] - sW[2] * rb[1], sV[1] + sW[2] * rb[0] - sW[0] * rb[2],
                           sV[2] + sW[0] * rb[1] - sW[1] * rb[0]};
            float uc = us[0] * cx(i) + us[1] * cy(i) + us[2] * cz(i);
            const float2 fr2 = ld2f<S>(fnew, L, i, m);
            float2 out2;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                float fr = c ? fr2.y : fr2.x;
                const float2 rm = ld_pair(rho, m);
                float C = 6.f * wgt(i) * (c ? rm.y : rm.x) * uc;
                (c ? out2.y : out2.x) = fr + C;
                float a = -(2.f * fr + C);  // F = (2 f* + C) c_ī, c_ī = -c_i
                float F[3] = {a * cx(i), a * cy(i), a * cz(i)};
                aF[0] += F[0];
                aF[1] += F[1];
                aF[2] += F[2];
                aT[0] += rb[1] * F[2] - rb[2] * F[1];
                aT[1] += rb[2] * F[0] - rb[0] * F[2];
                aT[2] += rb[0] * F[1] - rb[1] * F[0];
            }
            st2f<S>(fnew, L, i, m, out2);
        }
        for (int k2 = 0; k2 < 3; k2++) {
            acc[k2] += (double)aF[k2];
            acc[3 + k2] += (double)aT[k2];
        }
    }
    block_sum<6>(acc, red);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; k++) {
            P.Flink[3 * p + k] = acc[k];
            P.Tlink[3 * p + k] = acc[3 + k];
        }
    }
}

// ------------------------------------------------------------ link nodes
// For every particle node s of the step's link list and every direction j
// whose neighbour y = s + c_j is a fluid node (the link runs from y along
// c_i = -c_j into s): the fluid kernel reflected the post-collision
// f*_i(y) into slot j of y; add C = -6 w_i ρ^c(y) (u_surf·c_i) with u_surf =
// V + ω × r_b at the link midpoint r_b = s + c_j/2 - X (Eq. 4), and give
// the particle (2 f*_i + C) c_i and r_b × that (Eq. 5).  ρ^c(y) is the
// density kernel's, this step.  Force and torque are summed in 64-bit fixed
// point (2^-40 units): each FP32 link term is rounded once to an integer and
// integer additions are exact, so the totals do not depend on the order of
// the links.

// FP32 value to 64-bit fixed point in units of 2^-40 (two's complement in an
// unsigned word, so that wrap-around addition is exact); |v| is clamped to
// 2^22, far beyond any link term.
__device__ __forceinline__ unsigned long long to_fixed(float v)
{
    v = fminf(fmaxf(v, -4194304.f), 4194304.f);
    return (unsigned long long)__float2ll_rn(v * 1099511627776.f);
}

// Add this lane's sums v[6] for particle p (nothing for p < 0) to the
// particle's totals: lanes of the warp with the same particle are combined
// first (exact integer reductions over 16/16/32-bit limbs) and one lane per
// particle does the atomics.  Called by all 32 lanes.
__device__ __forceinline__ void warp_add_fix(int p, const unsigned long long v[6], unsigned long long *fix)
{
    const unsigned grp = __match_any_sync(0xffffffffu, p);
    const bool leader = (int)(threadIdx.x & 31) == __ffs(grp) - 1;
    unsigned long long tot[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const unsigned lo = (unsigned)v[k], hi = (unsigned)(v[k] >> 32);
        const unsigned s0 = __reduce_add_sync(grp, lo & 0xffffu);
        const unsigned s1 = __reduce_add_sync(grp, lo >> 16);
        const unsigned s2 = __reduce_add_sync(grp, hi);
        tot[k] = ((unsigned long long)s2 << 32) + ((unsigned long long)s1 << 16) + (unsigned long long)s0;
    }
    if (p < 0 || !leader) return;
#pragma unroll
    for (int k = 0; k < 6; k++) atomicAdd(&fix[6 * p + k], tot[k]);
}

// c_j for a direction j known only at run time (a lane's link): 2-bit
// fields c + 1 of the components, j = 0..18.
constexpr unsigned long long pack_dir(int axis)
{
    unsigned long long v = 0;
    for (int j = 0; j < Q; j++)
        v |= (unsigned long long)((axis == 0 ? cx(j) : (axis == 1 ? cy(j) : cz(j))) + 1) << (2 * j);
    return v;
}
constexpr unsigned long long CXP = pack_dir(0), CYP = pack_dir(1), CZP = pack_dir(2);
__device__ __forceinline__ int cdir(unsigned long long pack, int j) { return (int)((pack >> (2 * j)) & 3ull) - 1; }

// Per warp of the link kernels: the links of its 32 list entries in
// direction-major order, (entry lane, direction) per link.
struct LinkWarp {
    uint16_t desc[32 * (Q - 1)];
    unsigned bal[Q];
    int pre[Q];
};

// The links of 32 list entries (e = (node, mask of fluid neighbours) per
// lane; valid = false for a lane without an entry).  The entries' links
// are laid out direction by direction, so that lanes taking neighbouring
// links touch the same slot array at neighbouring nodes, and handed out 32
// at a time: every lane carries one link per round, and the loads of a
// round are all in flight together.  Called by all 32 lanes.
template <class S>
__device__ __forceinline__ void link_entries(const Lat &L, uint2 e, bool valid, const float *__restrict__ rho,
                                             const uint32_t *__restrict__ owner, const float4 *__restrict__ X32,
                                             const float4 *__restrict__ K32, unsigned long long *fix,
                                             typename S::P *fout, LinkWarp &w)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t fm = valid ? e.y : 0u;
    const int s = valid ? (int)e.x : 0;
    int p = -1;
    if (fm) {
        p = (int)owner[s];
        if ((unsigned)p >= (unsigned)L.np) {  // a particle node is always owned
            idx_ok(L, p, L.np, 20);
            p = -1;
            fm = 0;
        }
    }
    // direction j's links: the lanes of ballot j, after those of 1 .. j-1
    int total = 0;
#pragma unroll
    for (int j = 1; j < Q; j++) {
        const unsigned b = __ballot_sync(full, (fm >> j) & 1u);
        if (lane == j) {
            w.bal[j] = b;
            w.pre[j] = total;
        }
        total += __popc(b);
    }
    __syncwarp();
    for (uint32_t m = fm; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const int k = w.pre[j] + __popc(w.bal[j] & ((1u << lane) - 1u));
        w.desc[k] = (uint16_t)(lane | (j << 5));
    }
    __syncwarp();
    for (int k0 = 0; k0 < total; k0 += 32) {
        const int k = k0 + lane;
        const bool act = k < total;
        const int d = act ? w.desc[k] : 0;
        const int src = d & 31, j = act ? d >> 5 : 1;
        const int sn = __shfl_sync(full, s, src), pn = __shfl_sync(full, p, src);
        unsigned long long acc[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
        if (act) {
            const float4 X = X32[pn], V = K32[2 * pn], W = K32[2 * pn + 1];
            const int x = sn % L.nx, t = sn / L.nx, y = t % L.ny, z = t / L.ny;
            // sn - X, nearest image
            float dx = (float)x - X.x, dy = (float)y - X.y, dz = (float)z - X.z;
            if (dx > 0.5f * L.nx) dx -= L.nx;
            if (dx < -0.5f * L.nx) dx += L.nx;
            if (dy > 0.5f * L.ny) dy -= L.ny;
            if (dy < -0.5f * L.ny) dy += L.ny;
            if (!L.walls) {
                if (dz > 0.5f * L.nz) dz -= L.nz;
                if (dz < -0.5f * L.nz) dz += L.nz;
            }
            const int cxj = cdir(CXP, j), cyj = cdir(CYP, j), czj = cdir(CZP, j);
            int xn = x + cxj, yn = y + cyj, zn = z + czj;  // the fluid node
            xn = xn < 0 ? xn + L.nx : (xn >= L.nx ? xn - L.nx : xn);
            yn = yn < 0 ? yn + L.ny : (yn >= L.ny ? yn - L.ny : yn);
            zn = zn < 0 ? zn + L.nz : (zn >= L.nz ? zn - L.nz : zn);
            const int yf = xn + L.nx * (yn + L.ny * zn);
            const float fcx = (float)cxj, fcy = (float)cyj, fcz = (float)czj;
            const float rx = dx + 0.5f * fcx, ry = dy + 0.5f * fcy, rz = dz + 0.5f * fcz;
            // surface velocity V + ω × r_b at the link midpoint
            const float usx = __fsub_rn(__fmaf_rn(W.y, rz, V.x), __fmul_rn(W.z, ry));
            const float usy = __fsub_rn(__fmaf_rn(W.z, rx, V.y), __fmul_rn(W.x, rz));
            const float usz = __fsub_rn(__fmaf_rn(W.x, ry, V.z), __fmul_rn(W.y, rx));
            // u_surf·c_i with c_i = -c_j
            const float uci = -__fadd_rn(__fadd_rn(usx * fcx, usy * fcy), usz * fcz);
            const float w6 = j < 7 ? -6.f / 18.f : -6.f / 36.f;
            // both components of slot j of the fluid node: one pair access
            typename S::P *q = fout + pidx(L, j, yf);
            const float2 fs = ld2f<S>(fout, L, j, yf);
            const float2 ry2 = __ldg(reinterpret_cast<const float2 *>(rho) + yf);
            const float C0 = __fmul_rn(__fmul_rn(w6, ry2.x), uci);
            const float C1 = __fmul_rn(__fmul_rn(w6, ry2.y), uci);
            *q = S::enc2(make_float2(__fadd_rn(fs.x, C0) - L.base[0][j], __fadd_rn(fs.y, C1) - L.base[1][j]));
            float a = 0.f;
            a = __fadd_rn(a, __fmaf_rn(2.f, fs.x, C0));
            a = __fadd_rn(a, __fmaf_rn(2.f, fs.y, C1));
            // F = a c_i = -a c_j
            const float Fx = -a * fcx, Fy = -a * fcy, Fz = -a * fcz;
            acc[0] = to_fixed(Fx);
            acc[1] = to_fixed(Fy);
            acc[2] = to_fixed(Fz);
            acc[3] = to_fixed(__fsub_rn(__fmul_rn(ry, Fz), __fmul_rn(rz, Fy)));
            acc[4] = to_fixed(__fsub_rn(__fmul_rn(rz, Fx), __fmul_rn(rx, Fz)));
            acc[5] = to_fixed(__fsub_rn(__fmul_rn(rx, Fy), __fmul_rn(ry, Fx)));
        }
        warp_add_fix(act ? pn : -1, acc, fix);
    }
    __syncwarp();
}

// Warp-uniform trip count over the entries (every lane takes part in the
// reductions).
template <class S>
__device__ __forceinline__ void link_list(const Lat &L, const LinkList &ll, const float *rho, const uint32_t *owner,
                                          const Parts &P, typename S::P *fout, int first, int stride, LinkWarp &w)
{
    const int count = min(*ll.count, ll.cap);
    for (int w0 = first + (int)(threadIdx.x & ~31u); w0 < count; w0 += stride) {
        const int e = w0 + (threadIdx.x & 31);
        const bool valid = e < count;
        link_entries<S>(L, valid ? ll.ent[e] : make_uint2(0u, 0u), valid, rho, owner, P.X32, P.K32, P.fix, fout, w);
    }
}

template <class S>
__global__ void __launch_bounds__(256) k_link(Lat L, LinkList ll, const float *rho, const uint32_t *owner, Parts P,
                                              typename S::P *fout)
{
    __shared__ LinkWarp w[256 / 32];
    link_list<S>(L, ll, rho, owner, P, fout, blockIdx.x * blockDim.x, gridDim.x * blockDim.x, w[threadIdx.x >> 5]);
}

// Batched: blockIdx.y is the box; LINK_BATCH_CTAS CTAs per box.
constexpr int LINK_BATCH_CTAS = 4;

template <class S>
__global__ void __launch_bounds__(256) k_link_batch(BatchIndex B)
{
    const int b = blockIdx.y;
    const BoxDev &bx = B.box[b];
    if (!bx.links.ent || bx.P.n == 0) return;
    const int cur = B.par[2 * b], ocur = B.par[2 * b + 1];
    __shared__ LinkWarp w[256 / 32];
    link_list<S>(bx.L, bx.links, bx.rho, bx.owner[ocur], bx.P, (typename S::P *)bx.f[1 - cur],
                 blockIdx.x * blockDim.x, gridDim.x * blockDim.x, w[threadIdx.x >> 5]);
}

// --------------------------------------------------------- pair forces

__device__ __forceinline__ double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Anisotropic Hertz interaction (Eq. 6-8): φ = ε(ô_i,ô_j) (1 - r/σ)^{5/2}
// for r < σ with ε = ε̄ / sqrt(1 - χ^2 (ô_i·ô_j)^2), ε̄ = K_H σ̄^{5/2},
// σ̄ = 2 r_perp, and the Berne–Pechukas σ(ô_i, ô_j, r̂).  Returns σ; fills
// the force on j and the torques on i and j (minus the analytic gradients).
__device__ double hertz_bp(double K, double rp, double ro, const double r[3], const double oi[3],
                           const double oj[3], double fj[3], double ti[3], double tj[3])
{
    for (int k = 0; k < 3; k++) fj[k] = ti[k] = tj[k] = 0.0;
    double chi = (rp * rp - ro * ro) / (rp * rp + ro * ro);
    double sbar = 2.0 * ro;
    double rl = sqrt(dot3(r, r));
    if (!(rl > 0)) return sbar;
    double rh[3] = {r[0] / rl, r[1] / rl, r[2] / rl};
    double a = dot3(rh, oi), b = dot3(rh, oj), c = dot3(oi, oj);
    double ep = 1.0 + chi * c, em = 1.0 - chi * c;
    double S = (a + b) * (a + b) / ep + (a - b) * (a - b) / em;
    double D = 1.0 - 0.5 * chi * S;
    double sigma = sbar / sqrt(D);
    double s = rl / sigma;
    if (s >= 1.0) return sigma;
    double ebar = K * sbar * sbar * sqrt(sbar);
    double Ed = 1.0 - chi * chi * c * c;
    double eps = ebar / sqrt(Ed);
    double om = 1.0 - s;
    double phit = om * om * sqrt(om);
    double dphit = -2.5 * om * sqrt(om);
    double dsig_dS = 0.25 * chi * sbar / (D * sqrt(D));
    double dS_da = 2.0 * (a + b) / ep + 2.0 * (a - b) / em;
    double dS_db = 2.0 * (a + b) / ep - 2.0 * (a - b) / em;
    double dS_dc = -chi * (a + b) * (a + b) / (ep * ep) + chi * (a - b) * (a - b) / (em * em);
    double deps_dc = ebar * chi * chi * c / (Ed * sqrt(Ed));
    double gs = eps * dphit * (-rl / (sigma * sigma)) * dsig_dS;
    double dphi_drl = eps * dphit / sigma;
    double gi[3], gj[3];
    for (int k = 0; k < 3; k++) {
        double grad = dphi_drl * rh[k] + gs * (dS_da * (oi[k] - a * rh[k]) / rl + dS_db * (oj[k] - b * rh[k]) / rl);
        fj[k] = -grad;
        gi[k] = phit * deps_dc * oj[k] + gs * (dS_da * rh[k] + dS_dc * oj[k]);
        gj[k] = phit * deps_dc * oi[k] + gs * (dS_db * rh[k] + dS_dc * oi[k]);
    }
    double u[3];
    cross3(oi, gi, u);
    for (int k = 0; k < 3; k++) ti[k] = -u[k];
    cross3(oj, gj, u);
    for (int k = 0; k < 3; k++) tj[k] = -u[k];
    return sigma;
}

// The Hertz and lubrication (Eq. 9 with 2R -> σ, R^2 -> (σ/2)^2, only for
// gaps 0 < r - σ < Δc, opposing the normal approach) contribution of
// partner j to particle i.  The lubrication coefficient K (1/h - 1/Δc) is
// capped at the pair's reduced mass M_i M_j / (M_i + M_j): at the cap one
// update (Δt = 1) removes the normal approach speed; above it the explicit
// update would reverse the approach with growing speed as h -> 0.  A pair
// is evaluated in FP64 only when the FP32 distance of the centres is within
// reach_i + reach_j + Δc (+0.05 for the FP32 error).

__device__ void pair_term(const Lat &L, const Parts &P, const Pair &pp, int i, int j, const double oi[3],
                          double F[3], double T[3])
{
    int a = i < j ? i : j, b = i < j ? j : i;  // the pair is taken as (a, b), a < b
    double r[3];
    for (int k = 0; k < 3; k++) r[k] = pair_disp(L, k, P.X[3 * a + k], P.X[3 * b + k]);
    double Rj[3][3];
    rotmat(P.q + 4 * j, Rj);
    double oj[3] = {Rj[0][0], Rj[1][0], Rj[2][0]};
    const double *oa = i < j ? oi : oj, *ob = i < j ? oj : oi;
    double rp = 0.5 * (P.rp[a] + P.rp[b]), ro = 0.5 * (P.ro[a] + P.ro[b]);
    double fb[3], ta[3], tb[3];
    double sigma = hertz_bp(pp.k_hertz, rp, ro, r, oa, ob, fb, ta, tb);
    for (int k = 0; k < 3; k++) {
        F[k] += i == b ? fb[k] : -fb[k];
        T[k] += i == a ? ta[k] : tb[k];
    }
    double rl = sqrt(dot3(r, r));
    double h = rl - sigma;
    if (pp.lub_cut > 0 && h > 0 && h < pp.lub_cut) {
        double rh[3] = {r[0] / rl, r[1] / rl, r[2] / rl};
        double du[3] = {P.V[3 * a] - P.V[3 * b], P.V[3 * a + 1] - P.V[3 * b + 1], P.V[3 * a + 2] - P.V[3 * b + 2]};
        double K = 3.0 * M_PI * pp.mu * sigma * sigma / 8.0;
        double gam = K * (1.0 / h - 1.0 / pp.lub_cut);
        const double mred = P.M[a] * P.M[b] / (P.M[a] + P.M[b]);
        if (gam > mred) gam = mred;
        double s = gam * dot3(rh, du);
        for (int k = 0; k < 3; k++) F[k] += i == a ? -s * rh[k] : s * rh[k];
    }
}

// FP32 prefilter of a pair (centres and reaches in xyzw): nearest-image
// distance within reach_i + reach_j + extra.  Pairs it drops contribute
// exactly zero, so it decides nothing but the work done.
__device__ __forceinline__ bool near_pair(float4 me, float4 o, const float nl[3], const float inv[3], bool per_z,
                                          float extra)
{
    float dx = o.x - me.x, dy = o.y - me.y, dz = o.z - me.z;
    dx = __fmaf_rn(-nl[0], rintf(dx * inv[0]), dx);
    dy = __fmaf_rn(-nl[1], rintf(dy * inv[1]), dy);
    if (per_z) dz = __fmaf_rn(-nl[2], rintf(dz * inv[2]), dz);
    const float reach = me.w + o.w + extra;
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz)) <= reach * reach;
}

// ---------------------------------------------------------------- cells
// Per step: count the particles of each cell, exclusive prefix over the
// cells (one CTA), place each particle's index, then each particle gathers
// the candidates of the 27 cells around its own (each cell once when an
// axis has fewer than 3 cells), keeps those the FP32 prefilter passes, and
// sums the pair terms in increasing partner index: the same terms in the
// same order as a loop over all partners, so the sums do not depend on the
// order the cells were filled in.

__device__ __forceinline__ int cell_axis(float x, float n, float inv, int nc, bool periodic)
{
    if (periodic) x -= n * floorf(x / n);
    int c = (int)(x * inv);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_count(Lat L, Parts P, Cells C)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const float4 x = P.X32[i];
    const int cx_ = cell_axis(x.x, (float)L.nx, C.inv[0], C.n[0], true);
    const int cy_ = cell_axis(x.y, (float)L.ny, C.inv[1], C.n[1], true);
    const int cz_ = cell_axis(x.z, (float)L.nz, C.inv[2], C.n[2], !L.walls);
    const int c = cx_ + C.n[0] * (cy_ + C.n[1] * cz_);
    C.cid[i] = c;
    atomicAdd(&C.count[c], 1);
}

// Exclusive prefix of the cell counts; one CTA of 1024 threads, each over a
// contiguous run of cells.
__global__ void __launch_bounds__(1024) k_cell_scan(Cells C)
{
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (C.ncell + 1023) / 1024;
    const int c0 = min(t * per, C.ncell), c1 = min(c0 + per, C.ncell);
    int s = 0;
    for (int c = c0; c < c1; c++) s += C.count[c];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan of the run sums
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int c = c0; c < c1; c++) {
        C.start[c] = run;
        C.fill[c] = 0;
        run += C.count[c];
    }
    if (t == 1023) C.start[C.ncell] = part[1023];
}

__global__ void k_cell_fill(Parts P, Cells C)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int c = C.cid[i];
    C.idx[C.start[c] + atomicAdd(&C.fill[c], 1)] = i;
}

constexpr int CAND_MAX = 96;  // candidates held per particle; beyond that a full scan

__global__ void __launch_bounds__(128) k_pairs(Lat L, Parts P, Pair pp, Cells C)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const float4 me = P.X32[i];
    const float nl[3] = {(float)L.nx, (float)L.ny, (float)L.nz};
    const float inv[3] = {1.f / nl[0], 1.f / nl[1], 1.f / nl[2]};
    const bool per_z = !L.walls;
    const float extra = (float)pp.lub_cut + 0.05f;
    int cand[CAND_MAX];
    int nc = 0;
    bool overflow = false;
    const int c0 = C.cid[i];
    const int ci[3] = {c0 % C.n[0], (c0 / C.n[0]) % C.n[1], c0 / (C.n[0] * C.n[1])};
    int lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        if (C.n[k] < 3) {  // every cell of the axis once
            lo[k] = 0;
            hi[k] = C.n[k] - 1;
        } else {
            lo[k] = ci[k] - 1;
            hi[k] = ci[k] + 1;
        }
    }
    for (int dz = lo[2]; dz <= hi[2]; dz++) {
        int z = dz;
        if (C.n[2] >= 3) {
            if (per_z)
                z = (z + C.n[2]) % C.n[2];
            else if (z < 0 || z >= C.n[2])
                continue;
        }
        for (int dy = lo[1]; dy <= hi[1]; dy++) {
            const int y = C.n[1] >= 3 ? (dy + C.n[1]) % C.n[1] : dy;
            for (int dx = lo[0]; dx <= hi[0]; dx++) {
                const int x = C.n[0] >= 3 ? (dx + C.n[0]) % C.n[0] : dx;
                const int c = x + C.n[0] * (y + C.n[1] * z);
                for (int k = C.start[c]; k < C.start[c + 1]; k++) {
                    const int j = C.idx[k];
                    if (j == i || !near_pair(me, P.X32[j], nl, inv, per_z, extra)) continue;
                    if (nc < CAND_MAX)
                        cand[nc++] = j;
                    else
                        overflow = true;
                }
            }
        }
    }
    double Ri[3][3];
    rotmat(P.q + 4 * i, Ri);
    const double oi[3] = {Ri[0][0], Ri[1][0], Ri[2][0]};
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    if (!overflow) {
        for (int a = 1; a < nc; a++) {  // insertion sort: increasing partner index
            const int v = cand[a];
            int b = a - 1;
            while (b >= 0 && cand[b] > v) {
                cand[b + 1] = cand[b];
                b--;
            }
            cand[b + 1] = v;
        }
        for (int a = 0; a < nc; a++) pair_term(L, P, pp, i, cand[a], oi, F, T);
    } else {  // very dense: every partner in index order
        for (int j = 0; j < P.n; j++)
            if (j != i && near_pair(me, P.X32[j], nl, inv, per_z, extra)) pair_term(L, P, pp, i, j, oi, F, T);
    }
    for (int k = 0; k < 3; k++) {
        P.ppart[(size_t)k * P.n + i] = F[k];
        P.ppart[(size_t)(3 + k) * P.n + i] = T[k];
    }
}

// ------------------------------------------------------------ integrate
// Leapfrog translation (V += F/M, X += V), explicit Euler of the body-frame
// Euler equations, q <- normalise(q ⊗ exp(ω_body/2)).  The total force is
// momentum exchange + pair forces + the fill/empty momentum of the last
// coverage update.

__device__ void qmul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

__device__ void rotate_by_body_omega(double q[4], const double wb[3])
{
    double h[3] = {0.5 * wb[0], 0.5 * wb[1], 0.5 * wb[2]};
    double hn = sqrt(dot3(h, h));
    double dq[4] = {1.0, 0.0, 0.0, 0.0};
    if (hn > 0) {
        double s = sin(hn) / hn;
        dq[0] = cos(hn);
        dq[1] = s * h[0];
        dq[2] = s * h[1];
        dq[3] = s * h[2];
    }
    double qn[4];
    qmul(q, dq, qn);
    double nn = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    for (int k = 0; k < 4; k++) q[k] = qn[k] / nn;
}

__device__ __forceinline__ void integrate_body(const Lat &L, const Parts &P, int mode, int p)
{
    double F[3], T[3];
    for (int k = 0; k < 3; k++) {
        // link sums: FP64 from the two-pass link kernel, or 2^-40 fixed point
        // from the fused kernel (the other one is zero)
        const double fl = P.Flink[3 * p + k] + (double)(long long)P.fix[6 * p + k] * FIXED_UNIT;
        const double tl = P.Tlink[3 * p + k] + (double)(long long)P.fix[6 * p + 3 + k] * FIXED_UNIT;
        P.fix[6 * p + k] = 0ull;
        P.fix[6 * p + 3 + k] = 0ull;
        double fp = 0.0, tp = 0.0;
        for (int sp = 0; sp < P.nsplit; sp++) {
            fp += P.ppart[((size_t)sp * 6 + k) * P.n + p];
            tp += P.ppart[((size_t)sp * 6 + 3 + k) * P.n + p];
        }
        P.Fpair[3 * p + k] = fp;
        P.Tpair[3 * p + k] = tp;
        F[k] = fl + fp + P.Fpend[3 * p + k];
        T[k] = tl + tp + P.Tpend[3 * p + k];
        P.F[3 * p + k] = F[k];
        P.T[3 * p + k] = T[k];
        P.Fpend[3 * p + k] = 0.0;
        P.Tpend[3 * p + k] = 0.0;
        P.Flink[3 * p + k] = 0.0;
        P.Tlink[3 * p + k] = 0.0;
        P.Xold[3 * p + k] = P.X[3 * p + k];
    }
    double q[4];
    for (int k = 0; k < 4; k++) q[k] = P.qold[4 * p + k] = P.q[4 * p + k];
    if (mode == LBE_PARTICLES_STATIC) return;
    double X[3], V[3], W[3];
    for (int k = 0; k < 3; k++) {
        X[k] = P.X[3 * p + k];
        V[k] = P.V[3 * p + k];
        W[k] = P.W[3 * p + k];
    }
    double R[3][3];
    rotmat(q, R);
    double wb[3];
    for (int k = 0; k < 3; k++) wb[k] = R[0][k] * W[0] + R[1][k] * W[1] + R[2][k] * W[2];
    if (mode == LBE_PARTICLES_PRESCRIBED) {
        for (int k = 0; k < 3; k++) X[k] += V[k];
        rotate_by_body_omega(q, wb);
    } else {
        double M = P.M[p];
        for (int k = 0; k < 3; k++) {
            V[k] += F[k] / M;
            X[k] += V[k];
        }
        double tb[3];
        for (int k = 0; k < 3; k++) tb[k] = R[0][k] * T[0] + R[1][k] * T[1] + R[2][k] * T[2];
        double I[3] = {P.Ipar[p], P.Iperp[p], P.Iperp[p]};
        double Lb[3] = {I[0] * wb[0], I[1] * wb[1], I[2] * wb[2]};
        double wl[3];
        cross3(wb, Lb, wl);
        for (int k = 0; k < 3; k++) wb[k] += (tb[k] - wl[k]) / I[k];
        rotate_by_body_omega(q, wb);
        rotmat(q, R);
        for (int k = 0; k < 3; k++) W[k] = R[k][0] * wb[0] + R[k][1] * wb[1] + R[k][2] * wb[2];
    }
    for (int k = 0; k < 3; k++) {
        if (periodic_dim(L, k)) {
            double n = (double)ext_of(L, k);
            if (X[k] < 0) X[k] += n;
            if (X[k] >= n) X[k] -= n;
        }
        P.X[3 * p + k] = X[k];
        P.V[3 * p + k] = V[k];
        P.W[3 * p + k] = W[k];
    }
    for (int k = 0; k < 4; k++) P.q[4 * p + k] = q[k];
    float4 x32 = P.X32[p];
    x32.x = (float)X[0];
    x32.y = (float)X[1];
    x32.z = (float)X[2];
    P.X32[p] = x32;
    P.K32[2 * p] = make_float4((float)V[0], (float)V[1], (float)V[2], 0.f);
    P.K32[2 * p + 1] = make_float4((float)W[0], (float)W[1], (float)W[2], 0.f);
}

__global__ void k_integrate(Lat L, Parts P, int mode)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n) return;
    integrate_body(L, P, mode, p);
}

// ---------------------------------------------------------------- claim
// Every non-wall node inside a particle is claimed with atomicMin, so a
// node inside several particles goes to the lowest index.

__device__ __forceinline__ void claim_body(const Lat &L, const Parts &P, int p, uint32_t *__restrict__ owner_new)
{
    const PGeom &G = reinterpret_cast<const PGeom2 *>(P.geo)[p].now;
    const Box &box = G.box;
    for_candidates(box, G.g, G.X, [&](int ux, int u1, int u2, bool valid) {
        if (!valid) return;
        const int u[3] = {ux, u1, u2};
        const int x = wrapi(ux, L.nx), y = wrapi(u1, L.ny), z = wrapi(u2, L.nz);
        if (is_wall_z(L, z)) return;
        float d32[3];
#pragma unroll
        for (int a = 0; a < 3; a++)
            d32[a] = box.full[a] ? (float)node_disp(L, a, a == 0 ? x : (a == 1 ? y : z), G.X[a])
                                 : (float)(u[a] - G.Xi[a]) - G.Xf[a];
        float q32;
        bool in = inside_q32(G.g, d32, q32);
        if (!in && q32 <= 1.001f) {
            double dx[3] = {box_disp(L, box, 0, u[0], x, G.X[0]), box_disp(L, box, 1, u[1], y, G.X[1]),
                            box_disp(L, box, 2, u[2], z, G.X[2])};
            in = inside_exact(G.g, dx);
        }
        int n = x + L.nx * (y + L.ny * z);
        if (in && idx_ok(L, n, L.N, 4)) atomicMin(owner_new + n, (uint32_t)p);
    });
}

__global__ void __launch_bounds__(PT) k_claim(Lat L, Parts P, uint32_t *__restrict__ owner_new)
{
    claim_body(L, P, blockIdx.x, owner_new);
}

// ------------------------------------------------------------ transition
// Compare the old and new ownership.  A node whose owner changed is handled
// by exactly one CTA: that of the lower of its old and new owner.
//  - newly covered: its fluid (mass and momentum Σ f c) goes to the particle;
//  - newly uncovered: f = f^eq(ρ̄^c, u_surf) with ρ̄^c the mean over
//    neighbours fluid before and after (ρ_ref if none); the particle loses
//    that momentum;  both through the pending force/torque.
// With placement != 0 (particles just added) nodes only change type.

template <class S>
__device__ __forceinline__ void transition_body(const Lat &L, const Parts &P, int p, typename S::P *__restrict__ f,
                                                uint8_t *__restrict__ type, const uint32_t *__restrict__ own_old,
                                                const uint32_t *__restrict__ own_new, int placement)
{
    __shared__ double red[6][PT / 32];
    const PGeom2 &G2 = reinterpret_cast<const PGeom2 *>(P.geo)[p];
    const Box &box = G2.uni;
    const Geo &gold = G2.old_.g, &gnew = G2.now.g;
    const double *sXo = G2.old_.X, *sXu = G2.Xu;
    const double sX[3] = {P.X[3 * p], P.X[3 * p + 1], P.X[3 * p + 2]};
    const double sV[3] = {P.V[3 * p], P.V[3 * p + 1], P.V[3 * p + 2]};
    const double sW[3] = {P.W[3 * p], P.W[3 * p + 1], P.W[3 * p + 2]};
    double acc[6] = {0, 0, 0, 0, 0, 0};
    // a node whose owner changed lies in the old or the new ellipsoid of the
    // lower of its owners: the candidates of the old, then those of the new
    // not already visited
    auto visit = [&](int x, int y, int z) {
        int n = x + L.nx * (y + L.ny * z);
        if (!idx_ok(L, n, L.N, 5)) return;
        uint32_t o = own_old[n], w = own_new[n];
        if (o == w) return;
        if (min(o, w) != (uint32_t)p) return;
        if (o == NONE) {
            type[n] = PART;
            if (placement) return;
            double mom[3] = {0, 0, 0};
#pragma unroll
            for (int c = 0; c < 2; c++)
#pragma unroll
                for (int i = 0; i < Q; i++) {
                    const float2 v2 = ld2f<S>(f, L, i, n);
                    float v = c ? v2.y : v2.x;
                    if (cx(i)) mom[0] += cx(i) * (double)v;
                    if (cy(i)) mom[1] += cy(i) * (double)v;
                    if (cz(i)) mom[2] += cz(i) * (double)v;
                }
            double r[3] = {node_disp(L, 0, x, sX[0]), node_disp(L, 1, y, sX[1]), node_disp(L, 2, z, sX[2])};
            double t[3];
            cross3(r, mom, t);
            for (int k2 = 0; k2 < 3; k2++) {
                acc[k2] += mom[k2];
                acc[3 + k2] += t[k2];
            }
        } else if (w == NONE) {
            type[n] = FLUID;
            if (placement) return;
            float sr0 = 0.f, sr1 = 0.f;
            int cnt = 0;
            for (int i = 1; i < Q; i++) {
                int m = nbr_node(L, x, y, z, i);
                if (m < 0 || !idx_ok(L, m, L.N, 6)) continue;
                int mz = m / (L.nx * L.ny);
                if (is_wall_z(L, mz) || own_old[m] != NONE || own_new[m] != NONE) continue;
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int j = 0; j < Q; j++) {
                    const float2 v2 = ld2f<S>(f, L, j, m);
                    a0 += v2.x;
                    a1 += v2.y;
                }
                sr0 += a0;
                sr1 += a1;
                cnt++;
            }
            float rb0 = cnt ? sr0 / cnt : (float)L.rho_ref[0];
            float rb1 = cnt ? sr1 / cnt : (float)L.rho_ref[1];
            double r[3] = {node_disp(L, 0, x, sX[0]), node_disp(L, 1, y, sX[1]), node_disp(L, 2, z, sX[2])};
            float us[3] = {(float)(sV[0] + sW[1] * r[2] - sW[2] * r[1]),
                           (float)(sV[1] + sW[2] * r[0] - sW[0] * r[2]),
                           (float)(sV[2] + sW[0] * r[1] - sW[1] * r[0])};
            float uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
            double mom[3] = {0, 0, 0};
            float fe2[2][Q];
#pragma unroll
            for (int c = 0; c < 2; c++) {
                float rc = c ? rb1 : rb0;
#pragma unroll
                for (int i = 0; i < Q; i++) {
                    float cu = cx(i) * us[0] + cy(i) * us[1] + cz(i) * us[2];
                    float fe = wgt(i) * rc * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
                    fe2[c][i] = fe;
                    if (cx(i)) mom[0] += cx(i) * (double)fe;
                    if (cy(i)) mom[1] += cy(i) * (double)fe;
                    if (cz(i)) mom[2] += cz(i) * (double)fe;
                }
            }
#pragma unroll
            for (int i = 0; i < Q; i++) st2f<S>(f, L, i, n, make_float2(fe2[0][i], fe2[1][i]));
            double t[3];
            cross3(r, mom, t);
            for (int k2 = 0; k2 < 3; k2++) {
                acc[k2] -= mom[k2];
                acc[3 + k2] -= t[k2];
            }
        }
    };
    // per row: the old span, then the new span's parts left and right of it
    for_segments<3>(
        box,
        [&](int u1, int u2, int *xs, int *xe) {
            int a0, b0, a1, b1;
            row_span(gold, sXo, box, u1, u2, a0, b0);
            row_span(gnew, sXu, box, u1, u2, a1, b1);
            xs[0] = a0;
            xe[0] = b0;
            xs[1] = a1;
            xe[1] = a0 <= b0 ? min(b1, a0 - 1) : b1;
            xs[2] = a0 <= b0 ? max(a1, b0 + 1) : 1;
            xe[2] = a0 <= b0 ? b1 : 0;
        },
        [&](int ux, int u1, int u2, bool valid) {
            if (valid) visit(wrapi(ux, L.nx), wrapi(u1, L.ny), wrapi(u2, L.nz));
        });
    if (placement) return;
    block_sum<6>(acc, red);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; k++) {
            P.Fpend[3 * p + k] = acc[k];
            P.Tpend[3 * p + k] = acc[3 + k];
        }
    }
}

// Compiled for eight CTAs per SM (64 registers): most candidates only
// compare two owner words, and the occupancy hides their latency; the
// rare fill and empty spill a few registers.
template <class S>
__global__ void __launch_bounds__(PT, 8) k_transition(Lat L, Parts P, typename S::P *__restrict__ f,
                                                   uint8_t *__restrict__ type,
                                                   const uint32_t *__restrict__ own_old,
                                                   const uint32_t *__restrict__ own_new,
                                                   int placement)
{
    transition_body<S>(L, P, blockIdx.x, f, type, own_old, own_new, placement);
}

// ---------------------------------------------------------------- reset
// Clear an ownership map over every particle's box (old geometry when
// use_old), so the map is all NONE again for the next claim.

__device__ __forceinline__ void reset_body(const Lat &L, const Parts &P, int p, int use_old,
                                           uint32_t *__restrict__ owner)
{
    // The map holds, over this particle's box, only nodes inside its
    // ellipsoid (its own) or inside other particles' (cleared by them), so
    // clearing its own candidates empties the map.
    const PGeom2 &G2 = reinterpret_cast<const PGeom2 *>(P.geo)[p];
    const PGeom &G = use_old ? G2.old_ : G2.now;
    for_candidates(G.box, G.g, G.X, [&](int ux, int u1, int u2, bool valid) {
        if (!valid) return;
        int n = wrapi(ux, L.nx) + L.nx * (wrapi(u1, L.ny) + L.ny * wrapi(u2, L.nz));
        if (idx_ok(L, n, L.N, 7)) owner[n] = NONE;
    });
}

__global__ void __launch_bounds__(PT) k_reset(Lat L, Parts P, int use_old, uint32_t *__restrict__ owner)
{
    reset_body(L, P, blockIdx.x, use_old, owner);
}

// ---------------------------------------------------------------- shell
// Shell fill (Eq. 10 and the colour rule) of the nodes particle p owns,
// over its candidate rows; its nodes with fluid neighbours enter the link
// list.  With the wall planes these are all the solid nodes a fluid node
// can see.
// The densities of the fluid neighbours come from the density kernel.
// A particle's link entries go into the list as one contiguous segment
// (collected in shared memory, then one reservation and a coalesced copy),
// so that the link kernel, which walks the list in order, handles the
// links of one particle together: their slots share cache lines.  Entries
// beyond the buffer (very large particles) are appended directly.
constexpr int SHELL_BUF = 1024;

__global__ void __launch_bounds__(PT) k_shell_particles(Lat L, Parts P, const float *__restrict__ rho,
                                                        float *__restrict__ psi, const uint8_t *__restrict__ type,
                                                        const uint32_t *__restrict__ owner, LinkList ll)
{
    __shared__ uint2 buf[SHELL_BUF];
    __shared__ int nbuf, base;
    const int p = blockIdx.x;
    const PGeom &G = reinterpret_cast<const PGeom2 *>(P.geo)[p].now;
    const Box &box = G.box;
    const Geo &geo = G.g;
    const double *sX = G.X;
    const float dr = (float)P.drho[p];
    if (threadIdx.x == 0) nbuf = 0;
    __syncthreads();
    for_candidates(box, geo, sX, [&](int ux, int u1, int u2, bool valid) {
        int n = 0;
        uint32_t fm = 0;
        if (valid) {
            const int x = wrapi(ux, L.nx), y = wrapi(u1, L.ny), z = wrapi(u2, L.nz);
            n = x + L.nx * (y + L.ny * z);
            if (owner[n] == (uint32_t)p)
                fm = shell_fill(L, rho, psi, type, n, dr, [&](int i) { return nbr_node(L, x, y, z, i); });
        }
        if (!ll.ent) return;
        const unsigned want = __ballot_sync(0xffffffffu, fm != 0);
        if (!want) return;
        const int lane = threadIdx.x & 31, leader = __ffs(want) - 1;
        int k0 = 0;
        if (lane == leader) k0 = atomicAdd(&nbuf, __popc(want));
        k0 = __shfl_sync(0xffffffffu, k0, leader);
        const int k = k0 + __popc(want & ((1u << lane) - 1u));
        const bool spill = fm != 0 && k >= SHELL_BUF;
        if (fm && !spill) buf[k] = make_uint2((unsigned)n, fm);
        append_links(ll, n, spill ? fm : 0u);
    });
    if (!ll.ent) return;
    __syncthreads();
    const int cnt = min(nbuf, SHELL_BUF);
    if (threadIdx.x == 0) base = cnt ? atomicAdd(ll.count, cnt) : 0;
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x)
        if (base + k < ll.cap) ll.ent[base + k] = buf[k];
}

// Shell fill of the wall planes z = 0 and nz - 1 (Δρ = 0), with the
// densities of the neighbouring planes' fluid nodes from the populations.
template <class S>
__global__ void k_shell_walls(Lat L, const typename S::P *__restrict__ f, float *__restrict__ psi,
                              const uint8_t *__restrict__ type)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nxy = L.nx * L.ny;
    if (k >= 2 * nxy) return;
    const int z = k < nxy ? 0 : L.nz - 1, r = k < nxy ? k : k - nxy;
    const int x = r % L.nx, y = r / L.nx;
    const int n = x + L.nx * (y + L.ny * z);
    if (type[n] != WALL) return;
    shell_fill_with(L, psi, type, n, 0.f, [&](int i) { return nbr_node(L, x, y, z, i); },
                    [&](int m) { return node_rho2<S>(f, L, m); });
}

// ------------------------------------------------------------- batched
// One launch for all boxes of a batch: a CTA (or thread) per particle of the
// batch, in box order; parities come from the batch's device state.

__global__ void __launch_bounds__(PT) k_claim_batch(BatchIndex B, int total)
{
    const int g = blockIdx.x;
    const int b = find_box(B.part0, B.nbox, g);
    const BoxDev &bx = B.box[b];
    if (bx.mode == LBE_PARTICLES_STATIC) return;
    claim_body(bx.L, bx.P, g - B.part0[b], bx.owner[1 - B.par[2 * b + 1]]);
}

template <class S>
__global__ void __launch_bounds__(PT) k_transition_batch(BatchIndex B, int total)
{
    const int g = blockIdx.x;
    const int b = find_box(B.part0, B.nbox, g);
    const BoxDev &bx = B.box[b];
    if (bx.mode == LBE_PARTICLES_STATIC) return;
    const int cur = B.par[2 * b], ocur = B.par[2 * b + 1];
    transition_body<S>(bx.L, bx.P, g - B.part0[b], (typename S::P *)bx.f[1 - cur], bx.type, bx.owner[ocur],
                       bx.owner[1 - ocur], 0);
}

__global__ void __launch_bounds__(PT) k_reset_batch(BatchIndex B, int total)
{
    const int g = blockIdx.x;
    const int b = find_box(B.part0, B.nbox, g);
    const BoxDev &bx = B.box[b];
    if (bx.mode == LBE_PARTICLES_STATIC) return;
    reset_body(bx.L, bx.P, g - B.part0[b], 1, bx.owner[B.par[2 * b + 1]]);
}

__global__ void k_geom_batch(BatchIndex B, int total)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int b = find_box(B.part0, B.nbox, g);
    const BoxDev &bx = B.box[b];
    if (bx.mode == LBE_PARTICLES_STATIC) return;
    geom_body(bx.L, bx.P, g - B.part0[b]);
}

__global__ void k_integrate_batch(BatchIndex B, int total)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int b = find_box(B.part0, B.nbox, g);
    const BoxDev &bx = B.box[b];
    integrate_body(bx.L, bx.P, bx.mode, g - B.part0[b]);
}

// Pair forces within each box: one thread per particle over its box's
// particles in index order (the same terms in the same order as the cell
// list of a lattice stepped alone).
__global__ void k_pairs_batch(BatchIndex B, int total)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int b = find_box(B.part0, B.nbox, g);
    const BoxDev &bx = B.box[b];
    const Lat &L = bx.L;
    const Parts &P = bx.P;
    const int i = g - B.part0[b];
    double Ri[3][3];
    rotmat(P.q + 4 * i, Ri);
    const double oi[3] = {Ri[0][0], Ri[1][0], Ri[2][0]};
    const float4 me = P.X32[i];
    const float nl[3] = {(float)L.nx, (float)L.ny, (float)L.nz};
    const float inv[3] = {1.f / nl[0], 1.f / nl[1], 1.f / nl[2]};
    const bool per_z = !L.walls;
    const float extra = (float)bx.pair.lub_cut + 0.05f;
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    for (int j = 0; j < P.n; j++)
        if (j != i && near_pair(me, P.X32[j], nl, inv, per_z, extra)) pair_term(L, P, bx.pair, i, j, oi, F, T);
    for (int k = 0; k < 3; k++) {
        P.ppart[(size_t)k * P.n + i] = F[k];
        P.ppart[(size_t)(3 + k) * P.n + i] = T[k];
    }
}

// End of a batched step: flip each box's parities.
__global__ void k_flip_batch(BatchIndex B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nbox) return;
    B.par[2 * b] ^= 1;
    if (B.box[b].P.n > 0 && B.box[b].mode != LBE_PARTICLES_STATIC) B.par[2 * b + 1] ^= 1;
    if (B.box[b].links.count) *B.box[b].links.count = 0;  // ready for the next step's list
}

// Orientation of the first particle of each box (zeros for a box without
// particles), for the host's per-box convergence checks.
__global__ void k_batch_quat(BatchIndex B, double *out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nbox) return;
    const Parts &P = B.box[b].P;
    for (int k = 0; k < 4; k++) out[4 * b + k] = P.n > 0 ? P.q[k] : 0.0;
}

#ifdef LBE_CHECK
// Checked builds: after each step the node types must agree with the
// ownership map (particle iff owned).
__global__ void k_verify(Lat L, const uint8_t *type, const uint32_t *owner)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    bool part = type[n] == PART, own = owner[n] != NONE;
    if (part && !own) idx_ok(L, -1 - (long long)n, 0, 10);
    if (own && !part) idx_ok(L, -1 - (long long)n, 0, 11);
}
#endif

}  // namespace

void launch_pairs_batch(const BatchIndex &B, int total, cudaStream_t s)
{
    if (total > 0) k_pairs_batch<<<(total + 127) / 128, 128, 0, s>>>(B, total);
}

void launch_integrate_batch(const BatchIndex &B, int total, cudaStream_t s)
{
    if (total > 0) k_integrate_batch<<<(total + 127) / 128, 128, 0, s>>>(B, total);
}

void launch_geom_batch(const BatchIndex &B, int total, cudaStream_t s)
{
    if (total > 0) k_geom_batch<<<(total + 127) / 128, 128, 0, s>>>(B, total);
}

void launch_claim_batch(const BatchIndex &B, int total, cudaStream_t s)
{
    if (total > 0) k_claim_batch<<<total, PT, 0, s>>>(B, total);
}

void launch_reset_batch(const BatchIndex &B, int total, cudaStream_t s)
{
    if (total > 0) k_reset_batch<<<total, PT, 0, s>>>(B, total);
}

void launch_batch_quat(const BatchIndex &B, double *out, cudaStream_t s)
{
    k_batch_quat<<<(B.nbox + 127) / 128, 128, 0, s>>>(B, out);
}

void launch_flip_batch(const BatchIndex &B, cudaStream_t s)
{
    k_flip_batch<<<(B.nbox + 127) / 128, 128, 0, s>>>(B);
}

void launch_verify(const Lat &L, const uint8_t *type, const uint32_t *owner, cudaStream_t s)
{
#ifdef LBE_CHECK
    k_verify<<<(L.N + 255) / 256, 256, 0, s>>>(L, type, owner);
#endif
}

#define LBE_DISPATCH(storage, CALL)                                   \
    do {                                                              \
        switch (storage) {                                            \
        case LBE_STORE_F16_OFS: { using S = StF16; CALL; } break;     \
        case LBE_STORE_BF16_OFS: { using S = StBF16; CALL; } break;   \
        default: { using S = StF32; CALL; } break;                    \
        }                                                             \
    } while (0)

void launch_links(int storage, const Lat &L, const Parts &P, void *fnew, const float *rho,
                  const uint8_t *type, const uint32_t *owner, cudaStream_t s)
{
    if (P.n == 0) return;
    LBE_DISPATCH(storage, (k_links<S><<<P.n, PT, 0, s>>>(L, P, (typename S::P *)fnew, rho, type, owner)));
}

void launch_pairs(const Lat &L, const Parts &P, const Pair &pp, const Cells &C, cudaStream_t s)
{
    if (P.n == 0) return;
    const int b = (P.n + 127) / 128;
    cudaMemsetAsync(C.count, 0, (size_t)C.ncell * sizeof(int), s);
    k_cell_count<<<b, 128, 0, s>>>(L, P, C);
    k_cell_scan<<<1, 1024, 0, s>>>(C);
    k_cell_fill<<<b, 128, 0, s>>>(P, C);
    k_pairs<<<b, 128, 0, s>>>(L, P, pp, C);
}

void launch_geom(const Lat &L, const Parts &P, cudaStream_t s)
{
    if (P.n == 0) return;
    k_geom<<<(P.n + 127) / 128, 128, 0, s>>>(L, P);
}

size_t geom_bytes_per_particle() { return sizeof(PGeom2); }

void launch_integrate(const Lat &L, const Parts &P, int mode, cudaStream_t s)
{
    if (P.n == 0) return;
    k_integrate<<<(P.n + 127) / 128, 128, 0, s>>>(L, P, mode);
}

void launch_claim(const Lat &L, const Parts &P, int, uint32_t *owner_new, cudaStream_t s)
{
    if (P.n == 0) return;
    k_claim<<<P.n, PT, 0, s>>>(L, P, owner_new);
}

void launch_transition(int storage, const Lat &L, const Parts &P, void *f, uint8_t *type,
                       const uint32_t *owner_old, const uint32_t *owner_new, int placement,
                       cudaStream_t s)
{
    if (P.n == 0) return;
    LBE_DISPATCH(storage, (k_transition<S><<<P.n, PT, 0, s>>>(L, P, (typename S::P *)f, type, owner_old,
                                                               owner_new, placement)));
}

void launch_transition_batch(int storage, const BatchIndex &B, int total, cudaStream_t s)
{
    if (total == 0) return;
    LBE_DISPATCH(storage, (k_transition_batch<S><<<total, PT, 0, s>>>(B, total)));
}

void launch_link(int storage, const Lat &L, const LinkList &ll, const float *rho, const uint32_t *owner,
                 const Parts &P, void *fout, cudaStream_t s)
{
    if (P.n == 0 || !ll.ent) return;
    int blocks = (L.N + 255) / 256;
    if (blocks > 8 * 152) blocks = 8 * 152;
    LBE_DISPATCH(storage, (k_link<S><<<blocks, 256, 0, s>>>(L, ll, rho, owner, P, (typename S::P *)fout)));
}

void launch_link_batch(int storage, const BatchIndex &B, cudaStream_t s)
{
    dim3 grid(LINK_BATCH_CTAS, B.nbox);
    LBE_DISPATCH(storage, (k_link_batch<S><<<grid, 256, 0, s>>>(B)));
}

void launch_shell_particles(const Lat &L, const Parts &P, const float *rho, float *psi, const uint8_t *type,
                            const uint32_t *owner, const LinkList &ll, cudaStream_t s)
{
    if (P.n == 0) return;
    k_shell_particles<<<P.n, PT, 0, s>>>(L, P, rho, psi, type, owner, ll);
}

void launch_shell_walls(int storage, const Lat &L, const void *f, float *psi, const uint8_t *type, cudaStream_t s)
{
    if (!L.walls) return;
    const int n = 2 * L.nx * L.ny;
    LBE_DISPATCH(storage, (k_shell_walls<S><<<(n + 255) / 256, 256, 0, s>>>(L, (const typename S::P *)f, psi, type)));
}

void launch_reset(const Lat &L, const Parts &P, int use_old, uint32_t *owner, cudaStream_t s)
{
    if (P.n == 0) return;
    k_reset<<<P.n, PT, 0, s>>>(L, P, use_old, owner);
}

}  // namespace lbe
