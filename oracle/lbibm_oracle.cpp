// FP64 CPU oracle for the D3Q19 + immersed-boundary blood-flow step.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark load this library.  It shares no code, no
// header and no table with the CUDA library: every step below is written out
// plainly, in the order the paper states it, in double precision, without
// blocking, fusion or reordering.
//
// Source: Gusenbauer et al., "A tunable cancer cell filter using magnetic
// beads: cellular and fluid dynamic simulations" (arXiv:1110.0995).
//   Sec. 2.1  lattice-Boltzmann equation with an external force term (D3Q19).
//   Sec. 2.2  immersed-boundary cycle: transmit velocity to IB points,
//             compute node forces, spread them with an approximate delta
//             function, advance fluid and points.
//   Sec. 2.3.1 membrane moduli K^S (stretching), K^B (bending), K^A_l / K^A_g
//             (local / global area) and K^V (volume).
//   Sec. 2.3.3 the global area and volume need every node of a cell.
//   Sec. 2.4  bounce-back walls, obstacle nodes, no inside/outside distinction.
//
// The paper prints no formula for f^eq, the forcing term, the delta function or
// the membrane forces.  The readings used here (standard second-order
// equilibrium, Guo forcing, halfway bounce-back, trilinear delta, Dupin-style
// neo-Hookean stretching, dihedral-angle bending energy, homocentric area
// forces, facet-normal volume forces, massless IB points advected with the
// interpolated velocity, or points with mass and a frictional coupling) are
// each stated at the function that implements them.
//
// Layouts: lattice node p = x + nx*(y + ny*z); populations f[i*N + p];
// vector fields SoA v[d*N + p]; IB node positions / forces AoS x[3*j + d].
// Compiled with -ffp-contract=off so that no multiply-add is fused.

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

namespace {

using std::atan2;
using std::sqrt;
using std::tanh;

// ---------------------------------------------------------------------------
// D3Q19 velocity set (Sec. 2.1: "D3Q19 (three dimensions with 19 discrete
// velocities)").  Weights are not printed in the paper; these are the standard
// isotropic ones (w0 = 1/3, axis 1/18, diagonal 1/36, c_s^2 = 1/3).  Opposite
// directions come in consecutive pairs (1,2), (3,4), ..., (17,18).
// ---------------------------------------------------------------------------
const int Q = 19;
const int EV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
const double WQ[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
const int OPP[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};

inline double val(double a) { return a; }

// ---------------------------------------------------------------------------
// Forward-mode dual number v + d eps (eps^2 = 0): running the simulation with
// one parameter seeded (d = 1) gives the exact derivative of every quantity
// with respect to that parameter alongside its value.  Reference gradient for
// the differentiable variant below; shares nothing with any adjoint.
// ---------------------------------------------------------------------------
struct Dual {
    double v = 0.0, d = 0.0;
    Dual() = default;
    Dual(double a) : v(a), d(0.0) {}
    Dual(double a, double b) : v(a), d(b) {}
};
inline double val(const Dual& a) { return a.v; }
inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual& a, const Dual& b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(const Dual& a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, const Dual& b) { return Dual(a + b.v, b.d); }
inline Dual operator-(const Dual& a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, const Dual& b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(const Dual& a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(const Dual& a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual sqrt(const Dual& a) {
    const double r = std::sqrt(a.v);
    return Dual(r, a.d / (2.0 * r));
}
inline Dual atan2(const Dual& y, const Dual& x) {
    return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v));
}
inline Dual tanh(const Dual& a) {
    const double t = std::tanh(a.v);
    return Dual(t, (1.0 - t * t) * a.d);
}

// ---------------------------------------------------------------------------
// Equilibrium (Sec. 2.1: f^eq depends on rho and u; form not printed).
// Reading: f_i^eq = w_i rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u].
// ---------------------------------------------------------------------------
template <class R>
void equilibrium(R rho, const R u[3], R feq[Q]) {
    R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        R eu = EV[i][0] * u[0] + EV[i][1] * u[1] + EV[i][2] * u[2];
        feq[i] = WQ[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

// ---------------------------------------------------------------------------
// Forcing term F_i of the LB equation (Sec. 2.1: "F_i is the external force
// exerted by the immersed objects on the fluid"; scheme not printed).
// Reading: Guo et al. (2002),
//   F_i = (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . g,
// used together with the velocity u = (sum_i f_i e_i + g/2) / rho.
// ---------------------------------------------------------------------------
template <class R>
void guo_source(double tau, const R u[3], const R g[3], R S[Q]) {
    double pre = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < Q; ++i) {
        R eu = EV[i][0] * u[0] + EV[i][1] * u[1] + EV[i][2] * u[2];
        R s = 0.0;
        for (int d = 0; d < 3; ++d)
            s = s + (3.0 * (EV[i][d] - u[d]) + 9.0 * eu * EV[i][d]) * g[d];
        S[i] = pre * WQ[i] * s;
    }
}

// ---------------------------------------------------------------------------
// Fluid lattice (Sec. 2.1, 2.4)
// ---------------------------------------------------------------------------
template <class R>
struct Fluid {
    int nx = 0, ny = 0, nz = 0;
    long n = 0;
    double tau = 1.0;
    double G[3] = {0, 0, 0};           // uniform body force density
    int per[3] = {1, 0, 0};            // periodic axes; others carry halfway walls
    double uw[2][3] = {{0, 0, 0}, {0, 0, 0}};  // y-low / y-high wall velocity (tests)
    std::vector<R> f, fn;              // populations, current and next
    std::vector<R> g;                  // IB force density spread this step
    std::vector<R> gext;               // optional static extra force density
    std::vector<uint8_t> solid;        // 1 = obstacle node
    std::vector<R> rho, u;             // moments of the last collision

    long idx(int x, int y, int z) const { return x + (long)nx * (y + (long)ny * z); }
};

template <class R>
void fluid_init(Fluid<R>& F, int nx, int ny, int nz) {
    F.nx = nx; F.ny = ny; F.nz = nz;
    F.n = (long)nx * ny * nz;
    F.f.assign((size_t)Q * F.n, R(0.0));
    F.fn.assign((size_t)Q * F.n, R(0.0));
    F.g.assign((size_t)3 * F.n, R(0.0));
    F.solid.assign((size_t)F.n, 0);
    F.rho.assign((size_t)F.n, R(1.0));
    F.u.assign((size_t)3 * F.n, R(0.0));
    for (int i = 0; i < Q; ++i)
        for (long p = 0; p < F.n; ++p) F.f[(size_t)i * F.n + p] = WQ[i];
}

// One LB time step, Sec. 2.1:
//   f_i(x + e_i, t + 1) = f_i(x, t) - (f_i - f_i^eq)/tau + F_i.
// Done literally: per fluid node compute rho and u, collide, then move the
// post-collision value along e_i ("propagation").  A link that ends outside the
// domain (non-periodic axis) or on an obstacle node is reflected back into the
// node it came from, reversed (Sec. 2.4: "at the boundary the direction of
// velocity is inverted"); reading: halfway bounce-back, wall half a link away.
// A moving y-wall adds Ladd's momentum term -6 w_i rho0 (e_i . u_w), rho0 = 1.
// The force density at every fluid node is g_IB + g_ext + G: there is no
// inside/outside distinction (Sec. 2.4).
template <class R>
void lb_step(Fluid<R>& F) {
    const long N = F.n;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < F.nz; ++z) {
        for (int y = 0; y < F.ny; ++y) {
            for (int x = 0; x < F.nx; ++x) {
                const long p = F.idx(x, y, z);
                if (F.solid[p]) {
                    for (int i = 0; i < Q; ++i) F.fn[(size_t)i * N + p] = F.f[(size_t)i * N + p];
                    F.rho[p] = 1.0;
                    for (int d = 0; d < 3; ++d) F.u[(size_t)d * N + p] = 0.0;
                    continue;
                }
                R fl[Q];
                for (int i = 0; i < Q; ++i) fl[i] = F.f[(size_t)i * N + p];
                R rho = 0.0;
                for (int i = 0; i < Q; ++i) rho = rho + fl[i];
                R mom[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < Q; ++i)
                    for (int d = 0; d < 3; ++d) mom[d] = mom[d] + EV[i][d] * fl[i];
                R g[3];
                for (int d = 0; d < 3; ++d) {
                    g[d] = F.g[(size_t)d * N + p] + F.G[d];
                    if (!F.gext.empty()) g[d] = g[d] + F.gext[(size_t)d * N + p];
                }
                R u[3];
                for (int d = 0; d < 3; ++d) u[d] = (mom[d] + 0.5 * g[d]) / rho;
                R feq[Q], S[Q];
                equilibrium(rho, u, feq);
                guo_source(F.tau, u, g, S);
                F.rho[p] = rho;
                for (int d = 0; d < 3; ++d) F.u[(size_t)d * N + p] = u[d];
                for (int i = 0; i < Q; ++i) {
                    R post = fl[i] - (fl[i] - feq[i]) / F.tau + S[i];
                    int c[3] = {x + EV[i][0], y + EV[i][1], z + EV[i][2]};
                    const int dim[3] = {F.nx, F.ny, F.nz};
                    bool blocked = false;
                    int wall = -1;
                    for (int d = 0; d < 3; ++d) {
                        if (c[d] < 0 || c[d] >= dim[d]) {
                            if (F.per[d]) {
                                c[d] = (c[d] + dim[d]) % dim[d];
                            } else {
                                blocked = true;
                                if (d == 1 && wall < 0) wall = (c[d] < 0) ? 0 : 1;
                            }
                        }
                    }
                    if (!blocked && F.solid[F.idx(c[0], c[1], c[2])]) blocked = true;
                    if (blocked) {
                        R back = post;
                        if (wall >= 0) {
                            double eu = EV[i][0] * F.uw[wall][0] + EV[i][1] * F.uw[wall][1] +
                                        EV[i][2] * F.uw[wall][2];
                            back = back - 6.0 * WQ[i] * 1.0 * eu;
                        }
                        F.fn[(size_t)OPP[i] * N + p] = back;
                    } else {
                        F.fn[(size_t)i * N + F.idx(c[0], c[1], c[2])] = post;
                    }
                }
            }
        }
    }
    F.f.swap(F.fn);
}

// ---------------------------------------------------------------------------
// Immersed-boundary delta function (Sec. 2.2, steps 1 and 3: "discrete
// approximate delta-function"; kernel not printed).  Reading: trilinear,
// w(x - X) = prod_d (1 - |x_d - X_d|) over the 8 lattice nodes of the cell
// containing X.  The same weights transmit velocity (step 1) and spread force
// (step 3).  Nodes outside the domain on a non-periodic axis and obstacle nodes
// take no force and contribute zero velocity; weights are not renormalised.
// ---------------------------------------------------------------------------
template <class R>
struct Stencil {
    long node[8];
    R w[8];
    bool ok[8];
};

template <class R>
void stencil(const Fluid<R>& F, const R X[3], Stencil<R>& s) {
    const int dim[3] = {F.nx, F.ny, F.nz};
    long base[3];
    for (int d = 0; d < 3; ++d) base[d] = (long)std::floor(val(X[d]));
    for (int c = 0; c < 8; ++c) {
        long xc[3] = {base[0] + (c & 1), base[1] + ((c >> 1) & 1), base[2] + ((c >> 2) & 1)};
        R w = 1.0;
        bool ok = true;
        long ic[3];
        for (int d = 0; d < 3; ++d) {
            R dist = X[d] - (double)xc[d];
            if (val(dist) < 0) dist = -dist;
            w = w * (1.0 - dist);
            long v = xc[d];
            if (v < 0 || v >= dim[d]) {
                if (F.per[d]) v = ((v % dim[d]) + dim[d]) % dim[d];
                else ok = false;
            }
            ic[d] = v;
        }
        long p = ok ? F.idx((int)ic[0], (int)ic[1], (int)ic[2]) : -1;
        if (ok && F.solid[p]) ok = false;
        s.node[c] = p;
        s.w[c] = w;
        s.ok[c] = ok;
    }
}

template <class R>
void spread(const Fluid<R>& F, const R* X, const R* Fn, int n, R* g) {
    for (int j = 0; j < n; ++j) {
        Stencil<R> s;
        stencil(F, &X[3 * j], s);
        for (int c = 0; c < 8; ++c) {
            if (!s.ok[c]) continue;
            for (int d = 0; d < 3; ++d) g[(size_t)d * F.n + s.node[c]] = g[(size_t)d * F.n + s.node[c]] + s.w[c] * Fn[3 * j + d];
        }
    }
}

template <class R>
void interpolate(const Fluid<R>& F, const R* X, int n, const R* u, R* U) {
    for (int j = 0; j < n; ++j) {
        Stencil<R> s;
        stencil(F, &X[3 * j], s);
        R acc[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 8; ++c) {
            if (!s.ok[c]) continue;
            for (int d = 0; d < 3; ++d) acc[d] = acc[d] + s.w[c] * u[(size_t)d * F.n + s.node[c]];
        }
        for (int d = 0; d < 3; ++d) U[3 * j + d] = acc[d];
    }
}

// ---------------------------------------------------------------------------
// Membrane mechanics (Sec. 2.3.1)
// ---------------------------------------------------------------------------
template <class R>
inline void sub3(const R* a, const R* b, R* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
template <class R>
inline void cross3(const R* a, const R* b, R* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
template <class R>
inline R dot3(const R* a, const R* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Edge list of a closed oriented triangle mesh: every undirected edge {a,b}
// with the triangle (a,b,c) that traverses it as a->b and the triangle (b,a,d)
// that traverses it as b->a.  Returns false for a mesh that is not a closed
// oriented 2-manifold.
struct Topology {
    int n = 0, nt = 0;
    std::vector<int> tri;                 // 3 * nt
    std::vector<int> ea, eb, ec, ed;      // per edge
};

bool build_topology(const int* tri, int nt, int n, Topology& T) {
    T.n = n; T.nt = nt;
    T.tri.assign(tri, tri + 3 * nt);
    std::map<std::pair<int, int>, int> third;
    for (int t = 0; t < nt; ++t) {
        int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        for (int k = 0; k < 3; ++k) {
            if (v[k] < 0 || v[k] >= n) return false;
            std::pair<int, int> key(v[k], v[(k + 1) % 3]);
            if (key.first == key.second) return false;
            if (third.count(key)) return false;   // directed edge used twice
            third[key] = v[(k + 2) % 3];
        }
    }
    for (auto& kv : third) {
        int a = kv.first.first, b = kv.first.second;
        auto rev = third.find(std::make_pair(b, a));
        if (rev == third.end()) return false;     // open boundary
        if (a < b) {
            T.ea.push_back(a); T.eb.push_back(b);
            T.ec.push_back(kv.second); T.ed.push_back(rev->second);
        }
    }
    return true;
}

// Dihedral angle at edge (a,b) between triangle (a,b,c) and triangle (b,a,d),
// signed about the edge direction: theta = atan2((n1 x n2).e_hat, n1.n2).
template <class R>
R dihedral(const R* xa, const R* xb, const R* xc, const R* xd) {
    R e[3], ac[3], ba[3], bd[3], n1[3], n2[3], m[3];
    sub3(xb, xa, e); sub3(xc, xa, ac); sub3(xa, xb, ba); sub3(xd, xb, bd);
    cross3(e, ac, n1);
    cross3(ba, bd, n2);
    cross3(n1, n2, m);
    R le = sqrt(dot3(e, e));
    return atan2(dot3(m, e) / le, dot3(n1, n2));
}

template <class R>
R tri_area(const R* xa, const R* xb, const R* xc) {
    R ab[3], ac[3], n[3];
    sub3(xb, xa, ab); sub3(xc, xa, ac); cross3(ab, ac, n);
    return 0.5 * sqrt(dot3(n, n));
}

// Enclosed volume of a closed outward mesh: V = sum_t x_a . (x_b x x_c) / 6.
// Surface area: S = sum_t S_t.  (Sec. 2.3.3: both need every node of a cell.)
template <class R>
void area_volume(const R* x, const Topology& T, R& S, R& V) {
    S = 0.0; V = 0.0;
    for (int t = 0; t < T.nt; ++t) {
        const R* a = &x[3 * T.tri[3 * t]];
        const R* b = &x[3 * T.tri[3 * t + 1]];
        const R* c = &x[3 * T.tri[3 * t + 2]];
        R bc[3];
        cross3(b, c, bc);
        V = V + dot3(a, bc) / 6.0;
        S = S + tri_area(a, b, c);
    }
}

struct Rest {
    std::vector<double> L0, th0, S0t;
    double S0 = 0, V0 = 0;
};

void rest_state(const double* x0, const Topology& T, Rest& r) {
    size_t ne = T.ea.size();
    r.L0.resize(ne); r.th0.resize(ne); r.S0t.resize(T.nt);
    for (size_t e = 0; e < ne; ++e) {
        double d[3];
        sub3(&x0[3 * T.eb[e]], &x0[3 * T.ea[e]], d);
        r.L0[e] = std::sqrt(dot3(d, d));
        r.th0[e] = dihedral(&x0[3 * T.ea[e]], &x0[3 * T.eb[e]], &x0[3 * T.ec[e]], &x0[3 * T.ed[e]]);
    }
    for (int t = 0; t < T.nt; ++t)
        r.S0t[t] = tri_area(&x0[3 * T.tri[3 * t]], &x0[3 * T.tri[3 * t + 1]], &x0[3 * T.tri[3 * t + 2]]);
    area_volume(x0, T, r.S0, r.V0);
}

enum { TERM_STRETCH = 1, TERM_BEND = 2, TERM_AREA_LOCAL = 4, TERM_AREA_GLOBAL = 8, TERM_VOLUME = 16, TERM_ALL = 31 };

// Stretching, K^S (Sec. 2.3.1: nonlinear, "resembles a neo-Hookean
// behavior"; formula not printed).  Reading (Dupin et al. 2007 neo-Hookean
// bond): with lambda = L / L0,
//   T(lambda) = ks * kappa(lambda) * (lambda - 1),
//   kappa(lambda) = (lambda^(1/2) + lambda^(-5/2)) / (lambda + lambda^(-3)),
// pulling both ends of a stretched edge together along the edge.
template <class R>
void force_stretch(const R* x, const Topology& T, const Rest& r, double ks, R* F) {
    for (size_t e = 0; e < T.ea.size(); ++e) {
        int a = T.ea[e], b = T.eb[e];
        R d[3];
        sub3(&x[3 * b], &x[3 * a], d);
        R L = sqrt(dot3(d, d));
        R lam = L / r.L0[e];
        R sl = sqrt(lam);
        R kappa = (sl + 1.0 / (lam * lam * sl)) / (lam + 1.0 / (lam * lam * lam));
        R tension = ks * kappa * (lam - 1.0);
        for (int k = 0; k < 3; ++k) {
            R fk = tension * d[k] / L;
            F[3 * a + k] = F[3 * a + k] + fk;
            F[3 * b + k] = F[3 * b + k] - fk;
        }
    }
}

// Bending, K^B (Sec. 2.3.1: a preferred angle between the two faces sharing
// an edge; the departure from it gives the force).  Reading: energy
// E = (kb/2) (theta - theta0)^2 per edge and F = -grad E, distributed to all
// four points of the two faces (which conserves momentum).  Gradient of the
// dihedral angle (Bridson et al. 2003): with e = x_b - x_a, l = |e|,
//   grad_c = -l n1/|n1|^2,  grad_d = -l n2/|n2|^2,
//   grad_a = -(1 - s_c) grad_c - (1 - s_d) grad_d,
//   grad_b = -s_c grad_c - s_d grad_d,   s_v = (x_v - x_a).e / l^2.
template <class R>
void force_bend(const R* x, const Topology& T, const Rest& r, double kb, R* F) {
    for (size_t e = 0; e < T.ea.size(); ++e) {
        int a = T.ea[e], b = T.eb[e], c = T.ec[e], d = T.ed[e];
        const R *xa = &x[3 * a], *xb = &x[3 * b], *xc = &x[3 * c], *xd = &x[3 * d];
        R theta = dihedral(xa, xb, xc, xd);
        R ev[3], ac[3], ad[3], ba[3], bd[3], n1[3], n2[3];
        sub3(xb, xa, ev); sub3(xc, xa, ac); sub3(xd, xa, ad); sub3(xa, xb, ba); sub3(xd, xb, bd);
        cross3(ev, ac, n1);
        cross3(ba, bd, n2);
        R l2 = dot3(ev, ev);
        R l = sqrt(l2);
        R n1s = dot3(n1, n1), n2s = dot3(n2, n2);
        R sc = dot3(ac, ev) / l2, sd = dot3(ad, ev) / l2;
        R coef = -kb * (theta - r.th0[e]);
        for (int k = 0; k < 3; ++k) {
            R gc = -l * n1[k] / n1s;
            R gd = -l * n2[k] / n2s;
            R ga = -(1.0 - sc) * gc - (1.0 - sd) * gd;
            R gb = -sc * gc - sd * gd;
            F[3 * a + k] = F[3 * a + k] + coef * ga;
            F[3 * b + k] = F[3 * b + k] + coef * gb;
            F[3 * c + k] = F[3 * c + k] + coef * gc;
            F[3 * d + k] = F[3 * d + k] + coef * gd;
        }
    }
}

// Area, K^A_l and K^A_g (Sec. 2.3.1: a force proportional to the change of
// area that homocentrically shrinks or expands the face, computed per triangle
// (local) and for the whole cell (global)).  Reading: on triangle t with
// centroid c_t and w_i = x_i - c_t,
//   F_i = -k * dA * (2 S_t / sum_j |w_j|^2) * w_i,
// with dA = (S_t - S0_t)/S0_t (local, k = kal) or (S - S0)/S0 (global, k = kag):
// along w_i (homocentric), with the virtual work of E = (k/2) dA^2 * S0 under a
// homocentric scaling of the face.
template <class R>
void force_area(const R* x, const Topology& T, const Rest& r, double kal, double kag, R S, int terms, R* F) {
    for (int t = 0; t < T.nt; ++t) {
        int v[3] = {T.tri[3 * t], T.tri[3 * t + 1], T.tri[3 * t + 2]};
        R St = tri_area(&x[3 * v[0]], &x[3 * v[1]], &x[3 * v[2]]);
        R cen[3];
        for (int k = 0; k < 3; ++k) cen[k] = (x[3 * v[0] + k] + x[3 * v[1] + k] + x[3 * v[2] + k]) / 3.0;
        R w[3][3];
        R ww = 0.0;
        for (int i = 0; i < 3; ++i) {
            sub3(&x[3 * v[i]], cen, w[i]);
            ww = ww + dot3(w[i], w[i]);
        }
        R coef = 0.0;
        if (terms & TERM_AREA_LOCAL) coef = coef - kal * (St - r.S0t[t]) / r.S0t[t];
        if (terms & TERM_AREA_GLOBAL) coef = coef - kag * (S - r.S0) / r.S0;
        coef = coef * 2.0 * St / ww;
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) F[3 * v[i] + k] = F[3 * v[i] + k] + coef * w[i][k];
    }
}

// Volume, K^V (Sec. 2.3.1: per facet a force proportional to the change of
// volume, distributed to the facet's three points).  Reading:
//   F_i += -kv (V - V0)/V0 * n_t / 6   for each vertex i of facet t,
// n_t the unnormalised outward normal; on a closed mesh this is exactly
// -grad of E = (kv/2) (V - V0)^2 / V0.
template <class R>
void force_volume(const R* x, const Topology& T, const Rest& r, double kv, R V, R* F) {
    R coef = -kv * (V - r.V0) / r.V0 / 6.0;
    for (int t = 0; t < T.nt; ++t) {
        int v[3] = {T.tri[3 * t], T.tri[3 * t + 1], T.tri[3 * t + 2]};
        R ab[3], ac[3], n[3];
        sub3(&x[3 * v[1]], &x[3 * v[0]], ab);
        sub3(&x[3 * v[2]], &x[3 * v[0]], ac);
        cross3(ab, ac, n);
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) F[3 * v[i] + k] = F[3 * v[i] + k] + coef * n[k];
    }
}

// All node forces of one cell (Sec. 2.2 step 2), the sum of the selected terms.
template <class R>
void membrane_forces(const R* x, const Topology& T, const Rest& r, const double mod[5], int terms, R* F) {
    for (int j = 0; j < 3 * T.n; ++j) F[j] = 0.0;
    R S, V;
    area_volume(x, T, S, V);
    if (terms & TERM_STRETCH) force_stretch(x, T, r, mod[0], F);
    if (terms & TERM_BEND) force_bend(x, T, r, mod[1], F);
    if (terms & (TERM_AREA_LOCAL | TERM_AREA_GLOBAL)) force_area(x, T, r, mod[2], mod[3], S, terms, F);
    if (terms & TERM_VOLUME) force_volume(x, T, r, mod[4], V, F);
}

// ---------------------------------------------------------------------------
// Coupled system (Sec. 2.2, the four-step cycle)
// ---------------------------------------------------------------------------
template <class R>
struct Cell {
    Topology T;
    Rest rest;
    double mod[5];
    std::vector<double> x0;
    std::vector<R> x, F, U;
    std::vector<R> V;   // point velocities (IB points with mass only)
};

template <class R>
struct System {
    Fluid<R> fl;
    std::vector<Cell<R>> cells;
    long steps = 0;
    double rep_k = 0.0, rep_dc = 0.0;   // soft-sphere repulsion (off when rep_k == 0)
    std::vector<double> spheres;         // cx, cy, cz, r per bead (for the repulsion)
    double ib_m = 0.0, ib_gamma = 0.0;   // IB points with mass m and drag gamma (massless when ib_m == 0)
};

// Collisions (Sec. 2.4: cells repel each other and the walls through a soft
// potential cut at an interaction radius; form and constants not printed).
// Reading: harmonic soft sphere, for a separation d below the cut-off d_c a
// force k (d_c - d) along the separation on the node, between
//   * nodes of different cells (equal and opposite; x minimum image when x is
//     periodic),
//   * a node and a bead surface (d = |x - c| - r, along x - c),
//   * a node and a wall of a non-periodic axis (walls half a link outside the
//     first and last node: d = y + 1/2 or (n - 1/2) - y).
// The bounded stiffness k keeps the explicit coupling stable.  Added to the
// membrane forces before spreading.
template <class R>
void repulsion(System<R>& s) {
    const double k = s.rep_k, dc = s.rep_dc;
    const Fluid<R>& F = s.fl;
    const int dim[3] = {F.nx, F.ny, F.nz};
    const int nc = (int)s.cells.size();
    // node - node of different cells (a cell pair is skipped when its bounding
    // spheres are farther apart than the cut-off)
    std::vector<double> cx(3 * nc), rad(nc);
    for (int a = 0; a < nc; ++a) {
        const auto& c = s.cells[a];
        double m[3] = {0, 0, 0};
        for (int j = 0; j < c.T.n; ++j)
            for (int d = 0; d < 3; ++d) m[d] += val(c.x[3 * j + d]) / c.T.n;
        double r2 = 0.0;
        for (int j = 0; j < c.T.n; ++j) {
            double q = 0.0;
            for (int d = 0; d < 3; ++d) q += (val(c.x[3 * j + d]) - m[d]) * (val(c.x[3 * j + d]) - m[d]);
            r2 = std::max(r2, q);
        }
        for (int d = 0; d < 3; ++d) cx[3 * a + d] = m[d];
        rad[a] = std::sqrt(r2);
    }
    auto min_image = [&](R& dx, int d) {
        if (F.per[d]) {
            const double L = dim[d];
            dx = dx - L * std::floor(val(dx) / L + 0.5);
        }
    };
    for (int a = 0; a < nc; ++a)
        for (int b = a + 1; b < nc; ++b) {
            double dd[3], q = 0.0;
            for (int d = 0; d < 3; ++d) {
                dd[d] = cx[3 * a + d] - cx[3 * b + d];
                if (F.per[d]) dd[d] -= dim[d] * std::floor(dd[d] / dim[d] + 0.5);
                q += dd[d] * dd[d];
            }
            if (std::sqrt(q) > rad[a] + rad[b] + dc + 1.0) continue;
            auto& A = s.cells[a];
            auto& B = s.cells[b];
            for (int i = 0; i < A.T.n; ++i)
                for (int j = 0; j < B.T.n; ++j) {
                    R dv[3];
                    for (int d = 0; d < 3; ++d) {
                        dv[d] = A.x[3 * i + d] - B.x[3 * j + d];
                        min_image(dv[d], d);
                    }
                    R d2 = dot3(dv, dv);
                    if (!(val(d2) < dc * dc) || !(val(d2) > 0.0)) continue;
                    R dist = sqrt(d2);
                    R f = k * (dc - dist) / dist;
                    for (int d = 0; d < 3; ++d) {
                        A.F[3 * i + d] = A.F[3 * i + d] + f * dv[d];
                        B.F[3 * j + d] = B.F[3 * j + d] - f * dv[d];
                    }
                }
        }
    // node - bead and node - wall
    const int ns = (int)s.spheres.size() / 4;
    for (auto& c : s.cells)
        for (int j = 0; j < c.T.n; ++j) {
            R* x = &c.x[3 * j];
            for (int b = 0; b < ns; ++b) {
                R dv[3];
                for (int d = 0; d < 3; ++d) {
                    dv[d] = x[d] - s.spheres[4 * b + d];
                    min_image(dv[d], d);
                }
                R d2 = dot3(dv, dv);
                const double rr = s.spheres[4 * b + 3] + dc;
                if (!(val(d2) < rr * rr) || !(val(d2) > 0.0)) continue;
                R dist = sqrt(d2);
                R gap = dist - s.spheres[4 * b + 3];
                R f = k * (dc - gap) / dist;
                for (int d = 0; d < 3; ++d) c.F[3 * j + d] = c.F[3 * j + d] + f * dv[d];
            }
            for (int d = 0; d < 3; ++d) {
                if (F.per[d]) continue;
                R lo = x[d] + 0.5, hi = (dim[d] - 0.5) - x[d];
                if (val(lo) < dc) c.F[3 * j + d] = c.F[3 * j + d] + k * (dc - lo);
                if (val(hi) < dc) c.F[3 * j + d] = c.F[3 * j + d] - k * (dc - hi);
            }
        }
}

// One cycle.  Sec. 2.2 lists: (1) velocity from the grid to the IB points,
// (2) node forces, (3) spreading with the delta function, (4) fluid and point
// motion.  Reading (massless IB points; Newton's m and a drag coefficient are
// not given): the points move with the interpolated velocity of the fluid
// update of the same cycle,
//   F^t = F(X^t); g^t = spread(F^t, X^t); fluid update -> u^t;
//   X^{t+1} = X^t + interp(u^t, X^t).
template <class R>
void system_step(System<R>& s) {
    Fluid<R>& F = s.fl;
    std::fill(F.g.begin(), F.g.end(), R(0.0));
    for (auto& c : s.cells) membrane_forces(c.x.data(), c.T, c.rest, c.mod, TERM_ALL, c.F.data());
    if (s.rep_k != 0.0) repulsion(s);
    for (auto& c : s.cells) spread(F, c.x.data(), c.F.data(), c.T.n, F.g.data());
    lb_step(F);
    for (auto& c : s.cells) {
        interpolate(F, c.x.data(), c.T.n, F.u.data(), c.U.data());
        for (int j = 0; j < 3 * c.T.n; ++j) c.x[j] = c.x[j] + c.U[j];
    }
    s.steps++;
}

// IB points with mass (Sec. 2.2: m d^2X/dt^2 = F; the coupling force comes
// from the motion of the point relative to the fluid).  Reading: a frictional
// coupling -gamma (V - U), with U the fluid velocity of the last collision
// interpolated at X, the fluid receiving the opposite impulse; the membrane
// and collision forces F act on the points only.  One step splits into a kick
// by F and a drift under the drag with U held, solved exactly:
//   V      = W + F / m                                (kick)
//   X(1)   = X + U + (V - U) p1,   p1 = (1 - e^{-a}) / a,  a = gamma / m
//   W(1)   = U + (V - U) e^{-a}                       (drift, exact)
//   J      = integral of gamma (V(t) - U) dt = gamma (V - U) p1 = m (V - W(1))
// W is the point velocity after the drift (the state carried between steps,
// zero at the start).  For gamma = 0 this is the symplectic kick-drift
// (leapfrog) step and nothing reaches the fluid; for m -> 0, J -> F and
// X(1) -> X + U + F / gamma (the massless cycle with the velocity of the
// previous collision).  The fluid gains sum J, the points m sum (W(1) - W) =
// sum (F - J) = -sum J: momentum is conserved.
struct DragCoef {
    double a, p1, E;
};

DragCoef drag_coefficients(double m, double gamma) {
    DragCoef c;
    c.a = gamma / m;
    const double a = c.a;
    c.E = std::exp(-a);
    if (a < 1e-3) c.p1 = 1.0 - a / 2.0 + a * a / 6.0 - a * a * a / 24.0 + a * a * a * a / 120.0;
    else c.p1 = -std::expm1(-a) / a;
    return c;
}

// One cycle with massive IB points:
//   F^t = F(X^t); U^t = interp(u of the last collision, X^t);
//   kick, exact drag drift, impulse J^t as above; g^t = spread(J^t, X^t);
//   fluid update; X^{t+1}, W^{t+1}.
template <class R>
void system_step_massive(System<R>& s) {
    Fluid<R>& F = s.fl;
    std::fill(F.g.begin(), F.g.end(), R(0.0));
    for (auto& c : s.cells) membrane_forces(c.x.data(), c.T, c.rest, c.mod, TERM_ALL, c.F.data());
    if (s.rep_k != 0.0) repulsion(s);
    const double m = s.ib_m, gam = s.ib_gamma;
    const DragCoef k = drag_coefficients(m, gam);
    std::vector<std::vector<R>> dX(s.cells.size());
    for (size_t ci = 0; ci < s.cells.size(); ++ci) {
        auto& c = s.cells[ci];
        interpolate(F, c.x.data(), c.T.n, F.u.data(), c.U.data());
        std::vector<R> J(3 * c.T.n);
        dX[ci].resize(3 * c.T.n);
        for (int j = 0; j < 3 * c.T.n; ++j) {
            const R U = c.U[j];
            const R V = c.V[j] + c.F[j] / m;
            J[j] = gam * (V - U) * k.p1;
            dX[ci][j] = U + (V - U) * k.p1;
            c.V[j] = U + (V - U) * k.E;
        }
        spread(F, c.x.data(), J.data(), c.T.n, F.g.data());
    }
    lb_step(F);
    for (size_t ci = 0; ci < s.cells.size(); ++ci) {
        auto& c = s.cells[ci];
        for (int j = 0; j < 3 * c.T.n; ++j) c.x[j] = c.x[j] + dX[ci][j];
    }
    s.steps++;
}

// Magnetic bead interaction (Sec. 2.5): the force on bead 2 from bead 1 with
// moments m1, m2, r = x2 - x1 and c = mu0 / (4 pi), as printed (its bracket is
// left open; closed after the last term):
//   F = 3c / |r|^5 [ (m1.r) m2 + (m2.r) m1 + (m1.m2) r - 5 (m1.r)(m2.r) r / |r|^2 ]
void dipole_force(const double* m1, const double* m2, const double* r, double c, double* F) {
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double rr = std::sqrt(r2);
    const double m1r = m1[0] * r[0] + m1[1] * r[1] + m1[2] * r[2];
    const double m2r = m2[0] * r[0] + m2[1] * r[1] + m2[2] * r[2];
    const double m12 = m1[0] * m2[0] + m1[1] * m2[1] + m1[2] * m2[2];
    const double pre = 3.0 * c / (r2 * r2 * rr);
    for (int d = 0; d < 3; ++d)
        F[d] = pre * (m1r * m2[d] + m2r * m1[d] + m12 * r[d] - 5.0 * m1r * m2r * r[d] / r2);
}

// Energy of the pair (for the pins only): U = c / |r|^3 [m1.m2 - 3 (m1.r)(m2.r) / |r|^2].
double dipole_energy(const double* m1, const double* m2, const double* r, double c) {
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double m1r = m1[0] * r[0] + m1[1] * r[1] + m1[2] * r[2];
    const double m2r = m2[0] * r[0] + m2[1] * r[1] + m2[2] * r[2];
    const double m12 = m1[0] * m2[0] + m1[1] * m2[1] + m1[2] * m2[2];
    return c / (r2 * std::sqrt(r2)) * (m12 - 3.0 * m1r * m2r / r2);
}

struct BeadParams {
    double c;          // mu0 / (4 pi)
    double radius;     // bead radius R
    double k;          // contact stiffness
    double mobility;   // velocity per unit force (overdamped friction)
    double dt;
    double box[3];
    int per[3];
};

// Forces on every bead: the dipole interaction of every other bead plus, for
// two beads closer than 2R, a contact force k (2R - d) along their separation
// (the paper adds collision forces without a form; reading: harmonic).  On a
// periodic axis the separation is the minimum image.
void bead_forces(const double* x, const double* m, int n, const BeadParams& p, double* F) {
    for (int i = 0; i < 3 * n; ++i) F[i] = 0.0;
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            if (a == b) continue;
            double r[3];
            for (int d = 0; d < 3; ++d) {
                r[d] = x[3 * b + d] - x[3 * a + d];
                if (p.per[d]) r[d] -= p.box[d] * std::floor(r[d] / p.box[d] + 0.5);
            }
            double f[3];
            dipole_force(&m[3 * a], &m[3 * b], r, p.c, f);
            const double dist = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            const double overlap = 2.0 * p.radius - dist;
            for (int d = 0; d < 3; ++d) {
                F[3 * b + d] += f[d];
                if (overlap > 0.0) F[3 * b + d] += p.k * overlap * r[d] / dist;
            }
        }
}

// Overdamped bead motion (the paper's friction): x += mobility F dt, every
// bead from the forces at the same positions; wrapped into the box on
// periodic axes.
void bead_relax(double* x, const double* m, int n, const BeadParams& p, int steps) {
    std::vector<double> F(3 * (size_t)n);
    for (int s = 0; s < steps; ++s) {
        bead_forces(x, m, n, p, F.data());
        for (int i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                double v = x[3 * i + d] + p.mobility * F[3 * i + d] * p.dt;
                if (p.per[d]) v -= p.box[d] * std::floor(v / p.box[d]);
                x[3 * i + d] = v;
            }
    }
}

// Obstacles (Sec. 2.4 and 2.5: bead chains fixed in space are boundary
// nodes).  A lattice node is solid iff it lies inside or on any sphere,
// |x - c|^2 <= r^2, evaluated in double from the float inputs.
void rasterise(const float* sph, int ns, int nx, int ny, int nz, uint8_t* solid) {
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                uint8_t s = 0;
                for (int k = 0; k < ns; ++k) {
                    double dx = (double)x - (double)sph[4 * k];
                    double dy = (double)y - (double)sph[4 * k + 1];
                    double dz = (double)z - (double)sph[4 * k + 2];
                    double r = (double)sph[4 * k + 3];
                    double d2 = dx * dx;
                    d2 = d2 + dy * dy;
                    d2 = d2 + dz * dz;
                    if (d2 <= r * r) { s = 1; break; }
                }
                solid[x + (long)nx * (y + (long)ny * z)] = s;
            }
}

// ---------------------------------------------------------------------------
// Differentiable variant: the gradient of a filter objective with respect to
// the bead centres and the objective cell's stretching and bending moduli.
// A solid bitmask is piecewise constant in a bead centre (its derivative is
// zero almost everywhere), so here the beads are a smooth solid fraction
//   phi_k(x) = 1/2 [1 - tanh((|x - c_k| - r_k) / delta)],
//   phi(x)   = 1 - prod_k (1 - phi_k(x))          (union of the beads),
// acting as a Brinkman force density g_B = -alpha phi rho u taken implicitly:
//   u = (sum_i f_i e_i + g / 2) / (rho (1 + alpha phi / 2)),
//   g_tot = g - alpha phi rho u   in the Guo source.
// With alpha = 2 a node with phi = 1 leaves the collision with momentum g/2.
// Walls stay halfway bounce-back; nothing is a bitmask obstacle.
// Readings (the paper treats beads as bounce-back nodes only): the form of
// phi, the union, alpha = 2 and delta = 0.5 lu are this variant's constants.
// Objective: J = mean x-coordinate of the objective cell's nodes after T
// cycles minus the same at t = 0.
// ---------------------------------------------------------------------------
template <class R>
void brinkman_phi(const Fluid<R>& F, const std::vector<R>& bead, double delta, std::vector<R>& phi) {
    const int nb = (int)bead.size() / 4;
    phi.assign((size_t)F.n, R(0.0));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < F.nz; ++z)
        for (int y = 0; y < F.ny; ++y)
            for (int x = 0; x < F.nx; ++x) {
                R prod = 1.0;
                for (int k = 0; k < nb; ++k) {
                    R dx = (double)x - bead[4 * k], dy = (double)y - bead[4 * k + 1], dz = (double)z - bead[4 * k + 2];
                    R d2 = dx * dx + dy * dy + dz * dz;
                    R dist = val(d2) > 0.0 ? sqrt(d2) : R(0.0);
                    R phik = 0.5 * (1.0 - tanh((dist - bead[4 * k + 3]) / delta));
                    prod = prod * (1.0 - phik);
                }
                phi[F.idx(x, y, z)] = 1.0 - prod;
            }
}

// One LB step of the differentiable variant: lb_step with the Brinkman term in
// place of obstacle nodes.
template <class R>
void lb_step_brinkman(Fluid<R>& F, const std::vector<R>& phi, double alpha) {
    const long N = F.n;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < F.nz; ++z) {
        for (int y = 0; y < F.ny; ++y) {
            for (int x = 0; x < F.nx; ++x) {
                const long p = F.idx(x, y, z);
                R fl[Q];
                for (int i = 0; i < Q; ++i) fl[i] = F.f[(size_t)i * N + p];
                R rho = 0.0;
                for (int i = 0; i < Q; ++i) rho = rho + fl[i];
                R mom[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < Q; ++i)
                    for (int d = 0; d < 3; ++d) mom[d] = mom[d] + EV[i][d] * fl[i];
                R g[3];
                for (int d = 0; d < 3; ++d) g[d] = F.g[(size_t)d * N + p] + F.G[d];
                R u[3], gt[3];
                const R den = rho * (1.0 + 0.5 * alpha * phi[p]);
                for (int d = 0; d < 3; ++d) u[d] = (mom[d] + 0.5 * g[d]) / den;
                for (int d = 0; d < 3; ++d) gt[d] = g[d] - alpha * phi[p] * rho * u[d];
                R feq[Q], S[Q];
                equilibrium(rho, u, feq);
                guo_source(F.tau, u, gt, S);
                F.rho[p] = rho;
                for (int d = 0; d < 3; ++d) F.u[(size_t)d * N + p] = u[d];
                for (int i = 0; i < Q; ++i) {
                    R post = fl[i] - (fl[i] - feq[i]) / F.tau + S[i];
                    int c[3] = {x + EV[i][0], y + EV[i][1], z + EV[i][2]};
                    const int dim[3] = {F.nx, F.ny, F.nz};
                    bool blocked = false;
                    for (int d = 0; d < 3; ++d)
                        if (c[d] < 0 || c[d] >= dim[d]) {
                            if (F.per[d]) c[d] = (c[d] + dim[d]) % dim[d];
                            else blocked = true;
                        }
                    if (blocked) F.fn[(size_t)OPP[i] * N + p] = post;
                    else F.fn[(size_t)i * N + F.idx(c[0], c[1], c[2])] = post;
                }
            }
        }
    }
    F.f.swap(F.fn);
}

struct DiffMesh {
    std::vector<double> x0;
    std::vector<int> tri;
    double mod[5];
};

struct DiffProblem {
    int nx, ny, nz;
    double tau, G[3];
    int per[3];
    std::vector<double> beads;   // cx, cy, cz, r per bead
    double alpha, delta;
    std::vector<DiffMesh> meshes;
};

enum { SEED_NONE = 0, SEED_BEAD = 1, SEED_KS = 2, SEED_KB = 3 };

// A parameter value carrying the seed direction (unit tangent) when R is Dual.
template <class R> R seeded(double v);
template <> double seeded<double>(double v) { return v; }
template <> Dual seeded<Dual>(double v) { return Dual(v, 1.0); }

// Run T cycles from rest (f = w) and return J; with R = Dual and one parameter
// seeded, J.d is dJ / d(parameter).  u_out / x_out (optional, R = double) take
// the last cycle's velocity and every mesh's final positions.
template <class R>
R diff_run(const DiffProblem& P, int steps, int obj, int seed_kind, int seed_index, double* u_out, double* x_out) {
    Fluid<R> F;
    fluid_init(F, P.nx, P.ny, P.nz);
    F.tau = P.tau;
    for (int d = 0; d < 3; ++d) { F.G[d] = P.G[d]; F.per[d] = P.per[d]; }
    std::vector<R> bead(P.beads.begin(), P.beads.end());
    if (seed_kind == SEED_BEAD) bead[4 * (seed_index / 3) + seed_index % 3] = seeded<R>(P.beads[4 * (seed_index / 3) + seed_index % 3]);
    std::vector<R> phi;
    brinkman_phi(F, bead, P.delta, phi);
    struct C {
        Topology T;
        Rest rest;
        double mod[5];
        std::vector<R> x, Fa, Fs, Fb, Ftot, U;
        R ks, kb;
    };
    std::vector<C> cells(P.meshes.size());
    for (size_t m = 0; m < P.meshes.size(); ++m) {
        const DiffMesh& dm = P.meshes[m];
        C& c = cells[m];
        const int n = (int)dm.x0.size() / 3;
        build_topology(dm.tri.data(), (int)dm.tri.size() / 3, n, c.T);
        rest_state(dm.x0.data(), c.T, c.rest);
        for (int k = 0; k < 5; ++k) c.mod[k] = dm.mod[k];
        c.x.assign(dm.x0.begin(), dm.x0.end());
        c.Fa.assign(3 * n, R(0.0)); c.Fs = c.Fa; c.Fb = c.Fa; c.Ftot = c.Fa; c.U = c.Fa;
        c.ks = dm.mod[0];
        c.kb = dm.mod[1];
        if ((int)m == obj && seed_kind == SEED_KS) c.ks = seeded<R>(dm.mod[0]);
        if ((int)m == obj && seed_kind == SEED_KB) c.kb = seeded<R>(dm.mod[1]);
    }
    for (int t = 0; t < steps; ++t) {
        std::fill(F.g.begin(), F.g.end(), R(0.0));
        for (auto& c : cells) {
            const int n = c.T.n;
            // area and volume terms with the stated moduli; stretching and
            // bending are linear in ks and kb: ks * F_stretch(1) + kb * F_bend(1)
            membrane_forces(c.x.data(), c.T, c.rest, c.mod, TERM_AREA_LOCAL | TERM_AREA_GLOBAL | TERM_VOLUME, c.Fa.data());
            std::fill(c.Fs.begin(), c.Fs.end(), R(0.0));
            std::fill(c.Fb.begin(), c.Fb.end(), R(0.0));
            force_stretch(c.x.data(), c.T, c.rest, 1.0, c.Fs.data());
            force_bend(c.x.data(), c.T, c.rest, 1.0, c.Fb.data());
            for (int j = 0; j < 3 * n; ++j) c.Ftot[j] = c.Fa[j] + c.ks * c.Fs[j] + c.kb * c.Fb[j];
            spread(F, c.x.data(), c.Ftot.data(), n, F.g.data());
        }
        lb_step_brinkman(F, phi, P.alpha);
        for (auto& c : cells) {
            interpolate(F, c.x.data(), c.T.n, F.u.data(), c.U.data());
            for (int j = 0; j < 3 * c.T.n; ++j) c.x[j] = c.x[j] + c.U[j];
        }
    }
    if (u_out)
        for (size_t k = 0; k < F.u.size(); ++k) u_out[k] = val(F.u[k]);
    if (x_out) {
        size_t o = 0;
        for (auto& c : cells)
            for (auto& v : c.x) x_out[o++] = val(v);
    }
    const C& co = cells[obj];
    const int n = co.T.n;
    R mx = 0.0;
    double mx0 = 0.0;
    for (int j = 0; j < n; ++j) {
        mx = mx + co.x[3 * j];
        mx0 += P.meshes[obj].x0[3 * j];
    }
    return mx / (double)n - mx0 / (double)n;
}

}  // namespace

// ===========================================================================
// C interface (double precision) used from Python through ctypes.
// ===========================================================================
extern "C" {

typedef System<double> OrSys;

int or_version(void) { return 1; }

void or_constants(int* e /*19x3*/, double* w /*19*/, int* opp /*19*/) {
    for (int i = 0; i < Q; ++i) {
        for (int d = 0; d < 3; ++d) e[3 * i + d] = EV[i][d];
        w[i] = WQ[i];
        opp[i] = OPP[i];
    }
}

void or_equilibrium(double rho, const double* u, double* feq) { equilibrium(rho, u, feq); }

void or_guo_source(double tau, const double* u, const double* g, double* S) { guo_source(tau, u, g, S); }

void or_rasterise_spheres(const float* sph, int ns, int nx, int ny, int nz, uint8_t* solid) {
    rasterise(sph, ns, nx, ny, nz, solid);
}

void* or_sys_create(int nx, int ny, int nz, double tau, const double* G, const int* per, const double* uw) {
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5)) return nullptr;
    OrSys* s = new OrSys();
    fluid_init(s->fl, nx, ny, nz);
    s->fl.tau = tau;
    for (int d = 0; d < 3; ++d) {
        s->fl.G[d] = G ? G[d] : 0.0;
        s->fl.per[d] = per ? per[d] : 0;
    }
    if (uw)
        for (int k = 0; k < 6; ++k) s->fl.uw[k / 3][k % 3] = uw[k];
    return s;
}

void or_sys_destroy(void* h) { delete (OrSys*)h; }

void or_sys_set_solid(void* h, const uint8_t* solid) {
    OrSys* s = (OrSys*)h;
    std::memcpy(s->fl.solid.data(), solid, (size_t)s->fl.n);
}

void or_sys_set_repulsion(void* h, double k, double dc, const double* spheres, int ns) {
    OrSys* s = (OrSys*)h;
    s->rep_k = k;
    s->rep_dc = dc;
    s->spheres.assign(spheres, spheres + 4 * ns);
}

void or_sys_set_extra_force(void* h, const double* g) {
    OrSys* s = (OrSys*)h;
    if (!g) { s->fl.gext.clear(); return; }
    s->fl.gext.assign(g, g + 3 * s->fl.n);
}

void or_sys_init_equilibrium(void* h, double rho, const double* u) {
    OrSys* s = (OrSys*)h;
    double feq[Q];
    equilibrium(rho, u, feq);
    for (int i = 0; i < Q; ++i)
        for (long p = 0; p < s->fl.n; ++p) s->fl.f[(size_t)i * s->fl.n + p] = feq[i];
    for (long p = 0; p < s->fl.n; ++p) {
        s->fl.rho[p] = rho;
        for (int d = 0; d < 3; ++d) s->fl.u[(size_t)d * s->fl.n + p] = s->fl.solid[p] ? 0.0 : u[d];
    }
}

void or_sys_get_f(void* h, double* f) {
    OrSys* s = (OrSys*)h;
    std::memcpy(f, s->fl.f.data(), sizeof(double) * Q * s->fl.n);
}

void or_sys_set_f(void* h, const double* f) {
    OrSys* s = (OrSys*)h;
    std::memcpy(s->fl.f.data(), f, sizeof(double) * Q * s->fl.n);
}

// rho and u of the last collision (the velocity the IB points were moved with).
void or_sys_get_fields(void* h, double* rho, double* u) {
    OrSys* s = (OrSys*)h;
    if (rho) std::memcpy(rho, s->fl.rho.data(), sizeof(double) * s->fl.n);
    if (u) std::memcpy(u, s->fl.u.data(), sizeof(double) * 3 * s->fl.n);
}

int or_sys_add_mesh(void* h, const double* x0, int n, const int* tri, int nt, const double* mod) {
    OrSys* s = (OrSys*)h;
    Cell<double> c;
    if (!build_topology(tri, nt, n, c.T)) return -1;
    c.x0.assign(x0, x0 + 3 * n);
    rest_state(x0, c.T, c.rest);
    if (!(c.rest.V0 > 0)) return -2;
    for (int k = 0; k < 5; ++k) c.mod[k] = mod[k];
    c.x.assign(x0, x0 + 3 * n);
    c.F.assign(3 * n, 0.0);
    c.U.assign(3 * n, 0.0);
    c.V.assign(3 * n, 0.0);
    s->cells.push_back(std::move(c));
    return (int)s->cells.size() - 1;
}

void or_sys_set_nodes(void* h, int m, const double* x) {
    OrSys* s = (OrSys*)h;
    auto& c = s->cells[m];
    std::memcpy(c.x.data(), x, sizeof(double) * 3 * c.T.n);
}

void or_sys_get_nodes(void* h, int m, double* x) {
    OrSys* s = (OrSys*)h;
    auto& c = s->cells[m];
    std::memcpy(x, c.x.data(), sizeof(double) * 3 * c.T.n);
}

// Node forces of the last completed step (the forces spread in it).
void or_sys_get_forces(void* h, int m, double* F) {
    OrSys* s = (OrSys*)h;
    auto& c = s->cells[m];
    std::memcpy(F, c.F.data(), sizeof(double) * 3 * c.T.n);
}

void or_sys_step(void* h, int n_steps) {
    OrSys* s = (OrSys*)h;
    for (int k = 0; k < n_steps; ++k) {
        if (s->ib_m > 0.0) system_step_massive(*s);
        else system_step(*s);
    }
}

// IB points with mass m > 0 and drag gamma >= 0 (m = 0: massless points);
// the carried velocities W start at zero.
int or_sys_set_dynamics(void* h, double m, double gamma) {
    OrSys* s = (OrSys*)h;
    if (!(m >= 0.0) || !(gamma >= 0.0) || !std::isfinite(m) || !std::isfinite(gamma)) return -1;
    s->ib_m = m;
    s->ib_gamma = gamma;
    for (auto& c : s->cells) c.V.assign(3 * c.T.n, 0.0);
    return 0;
}

void or_sys_get_velocities(void* h, int m, double* v) {
    OrSys* s = (OrSys*)h;
    auto& c = s->cells[m];
    if (c.V.empty()) {
        std::memset(v, 0, sizeof(double) * 3 * c.T.n);
        return;
    }
    std::memcpy(v, c.V.data(), sizeof(double) * 3 * c.T.n);
}

void or_dipole_force(const double* m1, const double* m2, const double* r, double c, double* F) {
    dipole_force(m1, m2, r, c, F);
}

double or_dipole_energy(const double* m1, const double* m2, const double* r, double c) {
    return dipole_energy(m1, m2, r, c);
}

static BeadParams bead_params(const double* pr, const int* per) {
    BeadParams p;
    p.c = pr[0];
    p.radius = pr[1];
    p.k = pr[2];
    p.mobility = pr[3];
    p.dt = pr[4];
    for (int d = 0; d < 3; ++d) {
        p.box[d] = pr[5 + d];
        p.per[d] = per[d];
    }
    return p;
}

// params: c, radius, k, mobility, dt, box[3]
void or_bead_forces(const double* x, const double* m, int n, const double* params, const int* per, double* F) {
    bead_forces(x, m, n, bead_params(params, per), F);
}

void or_bead_relax(double* x, const double* m, int n, const double* params, const int* per, int steps) {
    bead_relax(x, m, n, bead_params(params, per), steps);
}

void or_drag_coefficients(double m, double gamma, double* a_p1_E) {
    const DragCoef c = drag_coefficients(m, gamma);
    a_p1_E[0] = c.a;
    a_p1_E[1] = c.p1;
    a_p1_E[2] = c.E;
}

// Differentiable variant (see diff_run).
void* or_diff_create(int nx, int ny, int nz, double tau, const double* G, const int* per, int nb, const double* beads,
                     double alpha, double delta) {
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || nb < 0) return nullptr;
    DiffProblem* P = new DiffProblem();
    P->nx = nx; P->ny = ny; P->nz = nz; P->tau = tau;
    for (int d = 0; d < 3; ++d) { P->G[d] = G[d]; P->per[d] = per[d]; }
    P->beads.assign(beads, beads + 4 * nb);
    P->alpha = alpha;
    P->delta = delta;
    return P;
}

void or_diff_destroy(void* h) { delete (DiffProblem*)h; }

int or_diff_add_mesh(void* h, const double* x0, int n, const int* tri, int nt, const double* mod) {
    DiffProblem* P = (DiffProblem*)h;
    Topology T;
    if (!build_topology(tri, nt, n, T)) return -1;
    DiffMesh m;
    m.x0.assign(x0, x0 + 3 * n);
    m.tri.assign(tri, tri + 3 * nt);
    for (int k = 0; k < 5; ++k) m.mod[k] = mod[k];
    P->meshes.push_back(std::move(m));
    return (int)P->meshes.size() - 1;
}

// J after `steps` cycles; with seed_kind != 0 also dJ/d(parameter) in *dJ:
// seed_kind 1 = bead coordinate seed_index (3 k + axis), 2 = ks, 3 = kb of mesh obj.
double or_diff_run(void* h, int steps, int obj, int seed_kind, int seed_index, double* dJ) {
    DiffProblem* P = (DiffProblem*)h;
    if (seed_kind == SEED_NONE) {
        if (dJ) *dJ = 0.0;
        return diff_run<double>(*P, steps, obj, SEED_NONE, 0, nullptr, nullptr);
    }
    Dual J = diff_run<Dual>(*P, steps, obj, seed_kind, seed_index, nullptr, nullptr);
    if (dJ) *dJ = J.d;
    return J.v;
}

// Final velocity field (3 x N) and positions of every mesh (concatenated) after `steps` cycles.
double or_diff_state(void* h, int steps, int obj, double* u, double* x) {
    DiffProblem* P = (DiffProblem*)h;
    return diff_run<double>(*P, steps, obj, SEED_NONE, 0, u, x);
}

// The solid fraction field (N) of the variant.
void or_diff_phi(void* h, double* phi) {
    DiffProblem* P = (DiffProblem*)h;
    Fluid<double> F;
    F.nx = P->nx; F.ny = P->ny; F.nz = P->nz;
    F.n = (long)P->nx * P->ny * P->nz;
    std::vector<double> ph;
    brinkman_phi(F, P->beads, P->delta, ph);
    std::memcpy(phi, ph.data(), sizeof(double) * F.n);
}

// Standalone pieces used by the pin tests.
int or_mesh_area_volume(const double* x, int n, const int* tri, int nt, double* S, double* V) {
    Topology T;
    if (!build_topology(tri, nt, n, T)) return -1;
    area_volume(x, T, *S, *V);
    return 0;
}

int or_mesh_edges(const int* tri, int nt, int n, int* edges /*4*E or NULL*/, int* n_edges) {
    Topology T;
    if (!build_topology(tri, nt, n, T)) return -1;
    *n_edges = (int)T.ea.size();
    if (edges)
        for (size_t e = 0; e < T.ea.size(); ++e) {
            edges[4 * e] = T.ea[e]; edges[4 * e + 1] = T.eb[e];
            edges[4 * e + 2] = T.ec[e]; edges[4 * e + 3] = T.ed[e];
        }
    return 0;
}

int or_mesh_forces(const double* x, const double* x0, int n, const int* tri, int nt, const double* mod, int terms,
                   double* F) {
    Topology T;
    if (!build_topology(tri, nt, n, T)) return -1;
    Rest r;
    rest_state(x0, T, r);
    membrane_forces(x, T, r, mod, terms, F);
    return 0;
}

double or_dihedral(const double* xa, const double* xb, const double* xc, const double* xd) {
    return dihedral(xa, xb, xc, xd);
}

void or_spread(void* h, const double* X, const double* Fn, int n, double* g) {
    OrSys* s = (OrSys*)h;
    spread(s->fl, X, Fn, n, g);
}

void or_interpolate(void* h, const double* X, int n, const double* u, double* U) {
    OrSys* s = (OrSys*)h;
    interpolate(s->fl, X, n, u, U);
}

}  // extern "C"
