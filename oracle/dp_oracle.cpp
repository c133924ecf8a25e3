// FP64 CPU oracle for the Deep Potential energy / force / virial evaluation.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// definition that the CUDA library is checked against.  Only the tests, the
// smoke entry and the CPU-baseline leg of the benchmark may load it.  It shares
// no code, header, table or helper with the CUDA path.
//
// What it computes (the model of Section II-A and Fig. 1 of the paper, with the
// DeePMD smooth-edition formulas the paper cites):
//   1. neighbour set of atom i within r_c with periodic images, canonical order
//      (neighbour type, j, nx, ny, nz); brute force O(N^2 * images) or a cell list
//      (Section II-A: LAMMPS builds the neighbour list; cell-list prior art);
//   2. environment matrix row (s, s dx/r, s dy/r, s dz/r), s = sw(r)/r, with the
//      smoothed first column (Section II-A), normalised by davg / dstd of the centre
//      type;
//   3. embedding net G = N_{ti,tj}(s_hat): 1->25->50->100, tanh, residual where the
//      width doubles (concatenate [x, x]) or stays (x)  (Section II-A "embedding net");
//   4. T = (1/S) R_hat^T G (4 x 100) summed over all S neighbour slots, a padded
//      slot being the row of an absent neighbour (R_tilde = 0, normalised like any
//      row, i.e. a neighbour at r_c); descriptor D = T^T T[:, :16] (100 x 16);
//   5. fitting net per centre type 1600->240->240->240->1, tanh, residual on the
//      equal-width layers (Section II-A "fitting net", sizes Section IV);
//      E_i = out + e_bias[ti], E = sum_i E_i;
//   6. forces F = -dE/dx by a hand-written reverse pass (Fig. 1(b): force by
//      backward propagation); virial Xi = -sum g (x) d over pairs;
//   7. velocity-Verlet NVE (Section II-A: LAMMPS updates velocities and positions),
//      neighbour rebuild every k steps with a skin (Section IV: skin 2 A).
// Readings where the paper is silent are listed with the library's design notes:
// quintic switch, davg / dstd read from the weights (0 / 1 for untrained random
// weights, or the per-type environment statistics of oracle_env_stats), padded
// slots as zero rows before normalisation, constant normaliser S = sum(sel), one
// embedding net per (ti, tj), index-ordered neighbour list, overflow is an error.
//
// Compile: g++ -O3 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction
// so that the neighbour distance test is bit-reproducible).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double y) : v(x), d(y) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return {s, a.d / (2.0 * s)}; }
inline Dual tanh(Dual a) { double t = std::tanh(a.v); return {t, a.d * (1.0 - t * t)}; }
inline Dual cos(Dual a) { return {std::cos(a.v), -a.d * std::sin(a.v)}; }
inline Dual sin(Dual a) { return {std::sin(a.v), a.d * std::cos(a.v)}; }
// Second-order jets along one input: value, first and second derivative (chain rule written
// out); used to evaluate the embedding net and its first two derivatives at table nodes.
struct Jet2 {
  double v, d, dd;
  Jet2() : v(0), d(0), dd(0) {}
  Jet2(double x) : v(x), d(0), dd(0) {}
  Jet2(double x, double y, double z) : v(x), d(y), dd(z) {}
};
inline Jet2 operator+(Jet2 a, Jet2 b) { return {a.v + b.v, a.d + b.d, a.dd + b.dd}; }
inline Jet2 operator-(Jet2 a, Jet2 b) { return {a.v - b.v, a.d - b.d, a.dd - b.dd}; }
inline Jet2 operator*(Jet2 a, Jet2 b) {
  return {a.v * b.v, a.d * b.v + a.v * b.d, a.dd * b.v + 2.0 * a.d * b.d + a.v * b.dd};
}
inline Jet2& operator+=(Jet2& a, Jet2 b) { a = a + b; return a; }
inline Jet2 tanh(Jet2 a) {
  const double t = std::tanh(a.v), t1 = 1.0 - t * t;  // tanh' = 1 - t^2, tanh'' = -2 t (1 - t^2)
  return {t, t1 * a.d, t1 * a.dd - 2.0 * t * t1 * a.d * a.d};
}
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
inline double val(Jet2 a) { return a.v; }
using std::sqrt;
using std::tanh;
using std::cos;
using std::sin;

// ---------------------------------------------------------------- model
struct Sizes { int n1, n2, n3, m2, f1, f2, f3; };

template <class T>
struct Model {
  int ntypes = 0, switch_kind = 0;
  double rc = 0, rs = 0;
  Sizes sz{};
  std::vector<int> sel, sel_off;   // per neighbour type
  int S = 0;
  std::vector<T> theta;            // flat parameters in blob order
  std::vector<double> davg, dstd;  // [nt][4]
  // parameter block offsets
  std::vector<size_t> emb_off;     // [nt*nt]
  std::vector<size_t> fit_off;     // [nt]
  size_t ebias_off = 0, ntheta = 0;
  // Tabulated embedding (compressed model): when tab_n > 0 every embedding net is replaced by
  // a piecewise quintic in its input on tab_n uniform intervals of width tab_h from tab_x0,
  // coefficients tab[((pair * tab_n + i) * n3 + a) * 6 + p] of u^p, u = (x - x_i) / tab_h.
  int tab_n = 0;
  double tab_x0 = 0.0, tab_h = 0.0;
  std::vector<double> tab;
  // Nearest-first truncation: a neighbour type with more than sel_t neighbours within r_c keeps
  // its sel_t nearest instead of raising the overflow error.
  bool nearest = false;
  size_t emb_size() const { const Sizes& s = sz; return (size_t)s.n1 * 2 + (size_t)s.n1 * s.n2 + s.n2 + (size_t)s.n2 * s.n3 + s.n3; }
  size_t fit_size() const { const Sizes& s = sz; return (size_t)s.n3 * s.m2 * s.f1 + s.f1 + (size_t)s.f1 * s.f2 + s.f2 + (size_t)s.f2 * s.f3 + s.f3 + s.f3 + 1; }
};

struct Blob {
  const unsigned char* p; size_t n;
  template <class X> bool get(size_t off, X* out, size_t cnt = 1) const {
    if (off + sizeof(X) * cnt > n) return false;
    std::memcpy(out, p + off, sizeof(X) * cnt);
    return true;
  }
};

// Parse the weight blob (layout documented with the input generator).
bool load_model(const void* data, size_t nbytes, Model<double>& m) {
  Blob b{static_cast<const unsigned char*>(data), nbytes};
  char magic[4];
  int32_t ver, nt, sk;
  if (!b.get(0, magic, 4) || std::memcmp(magic, "DPW1", 4) != 0) return false;
  b.get(4, &ver); b.get(8, &nt); b.get(12, &sk);
  if (ver != 1 || nt < 1 || nt > 8) return false;
  m.ntypes = nt; m.switch_kind = sk;
  b.get(16, &m.rc); b.get(24, &m.rs);
  int32_t e[3], ax, f[3];
  b.get(32, e, 3); b.get(44, &ax); b.get(48, f, 3);
  m.sz = {e[0], e[1], e[2], ax, f[0], f[1], f[2]};
  size_t off = 64;
  std::vector<int32_t> sel(nt);
  b.get(off, sel.data(), nt);
  off += 4 * (size_t)(nt + (nt % 2));
  off += 8 * (size_t)nt;  // type names
  m.sel.assign(sel.begin(), sel.end());
  m.sel_off.resize(nt + 1);
  m.sel_off[0] = 0;
  for (int t = 0; t < nt; ++t) m.sel_off[t + 1] = m.sel_off[t] + m.sel[t];
  m.S = m.sel_off[nt];
  m.emb_off.resize(nt * nt);
  m.fit_off.resize(nt);
  size_t q = 0;
  for (int i = 0; i < nt * nt; ++i) { m.emb_off[i] = q; q += m.emb_size(); }
  for (int t = 0; t < nt; ++t) { m.fit_off[t] = q; q += m.fit_size(); }
  m.ebias_off = q; q += nt;
  m.ntheta = q;
  m.theta.resize(q);
  if (!b.get(off, m.theta.data(), q)) return false;
  off += 8 * q;
  m.davg.resize(nt * 4); m.dstd.resize(nt * 4);
  if (!b.get(off, m.davg.data(), nt * 4)) return false;
  off += 8 * nt * 4;
  if (!b.get(off, m.dstd.data(), nt * 4)) return false;
  return true;
}

template <class T>
Model<T> cast_model(const Model<double>& m) {
  Model<T> o;
  o.ntypes = m.ntypes; o.switch_kind = m.switch_kind; o.rc = m.rc; o.rs = m.rs; o.sz = m.sz;
  o.sel = m.sel; o.sel_off = m.sel_off; o.S = m.S; o.davg = m.davg; o.dstd = m.dstd;
  o.emb_off = m.emb_off; o.fit_off = m.fit_off; o.ebias_off = m.ebias_off; o.ntheta = m.ntheta;
  o.tab_n = m.tab_n; o.tab_x0 = m.tab_x0; o.tab_h = m.tab_h; o.tab = m.tab; o.nearest = m.nearest;
  o.theta.resize(m.theta.size());
  for (size_t i = 0; i < m.theta.size(); ++i) o.theta[i] = T(m.theta[i]);
  return o;
}

// ---------------------------------------------------------------- neighbour list
struct NList {
  int N = 0, S = 0;
  std::vector<int> j;     // [N*S], -1 = padding
  std::vector<int> img;   // [N*S] packed image code
  std::vector<int> count; // [N*nt] real neighbours per type (may exceed sel on overflow)
  bool overflow = false;
};

inline int pack_img(int nx, int ny, int nz) {
  return ((nx + 512) << 20) | ((ny + 512) << 10) | (nz + 512);
}
inline void unpack_img(int c, int& nx, int& ny, int& nz) {
  nx = ((c >> 20) & 1023) - 512; ny = ((c >> 10) & 1023) - 512; nz = (c & 1023) - 512;
}

// Wrap into [0, L): w = x - L*floor(x/L); a result on the boundary (w < 0 or w >= L,
// possible only through rounding) becomes 0.
inline double wrap1(double x, double L) {
  double t = std::floor(x / L);
  double p = t * L;
  double w = x - p;
  if (w < 0.0 || w >= L) w = 0.0;
  return w;
}

// Periodic cell: box vectors a, b, c as the rows of H (row-major [9]); an image n = (n0, n1, n2)
// of atom j sits at x_j + n H.  Orthorhombic when every off-diagonal entry is 0.
struct Box {
  double H[9];
  double Hinv[9];  // s = x Hinv (fractional coordinates, row vector)
  double L[3];     // diagonal (the edge lengths of an orthorhombic box)
  double w[3];     // perpendicular widths V / |b x c|, V / |c x a|, V / |a x b|
  bool tri;
};

// Component c of the image shift n H, in the fixed order ((n0 H0c + n1 H1c) + n2 H2c); for an
// orthorhombic box it equals n_c L_c exactly.
inline double shift(const Box& B, const int* n, int c) {
  double p0 = (double)n[0] * B.H[c];
  double p1 = (double)n[1] * B.H[3 + c];
  double p2 = (double)n[2] * B.H[6 + c];
  return (p0 + p1) + p2;
}

// Squared distance of (j, n) seen from i, in the fixed operation order
// dx = (x_j + (n H)_x) - x_i; r2 = ((dx*dx) + (dy*dy)) + (dz*dz).
inline double dist2(const double* xi, const double* xj, const int* n, const Box& B) {
  double r2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    double sh = shift(B, n, a);
    double p = xj[a] + sh;
    double d = p - xi[a];
    double dd = d * d;
    r2 = (a == 0) ? dd : r2 + dd;
  }
  return r2;
}

inline void frac(const Box& B, const double* x, double* s) {
  for (int c = 0; c < 3; ++c) {
    double p0 = x[0] * B.Hinv[c], p1 = x[1] * B.Hinv[3 + c], p2 = x[2] * B.Hinv[6 + c];
    s[c] = (p0 + p1) + p2;
  }
}

struct Cand { int t, j, img; double r2; };
inline bool cand_less(const Cand& a, const Cand& b) {
  if (a.t != b.t) return a.t < b.t;
  if (a.j != b.j) return a.j < b.j;
  return a.img < b.img;
}
// Distance rank for nearest-first truncation: r^2, then the canonical key (j, image).
inline bool cand_nearer(const Cand& a, const Cand& b) {
  if (a.r2 != b.r2) return a.r2 < b.r2;
  if (a.j != b.j) return a.j < b.j;
  return a.img < b.img;
}

// Nearest-first truncation of one atom's candidates (sorted canonically): every type with more
// than sel_t candidates keeps its sel_t nearest (cand_nearer), still in canonical order.
void keep_nearest(std::vector<Cand>& c, const std::vector<int>& sel, int nt) {
  std::vector<Cand> out;
  for (int t = 0; t < nt; ++t) {
    std::vector<Cand> ct;
    for (const Cand& x : c) if (x.t == t) ct.push_back(x);
    if ((int)ct.size() > sel[t]) {
      std::sort(ct.begin(), ct.end(), cand_nearer);
      ct.resize(sel[t]);
      std::sort(ct.begin(), ct.end(), cand_less);
    }
    out.insert(out.end(), ct.begin(), ct.end());
  }
  c.swap(out);
}

// Emit candidate list of atom i (already sorted) into the padded per-type layout.
void emit(NList& nl, int i, const std::vector<Cand>& c, const std::vector<int>& sel,
          const std::vector<int>& sel_off, int nt) {
  int* jrow = &nl.j[(size_t)i * nl.S];
  int* irow = &nl.img[(size_t)i * nl.S];
  for (int k = 0; k < nl.S; ++k) { jrow[k] = -1; irow[k] = 0; }
  std::vector<int> cnt(nt, 0);
  for (const Cand& x : c) {
    int k = cnt[x.t]++;
    if (k < sel[x.t]) { jrow[sel_off[x.t] + k] = x.j; irow[sel_off[x.t] + k] = x.img; }
  }
  for (int t = 0; t < nt; ++t) nl.count[(size_t)i * nt + t] = cnt[t];
}

// Brute force: every j and every image n in [-nmax, nmax]^3, nmax = ceil(rcut / L).
void nlist_brute(int N, const double* xw, const int* types, const Box& B, double rcut,
                 const std::vector<int>& sel, NList& nl, bool nearest = false) {
  int nt = (int)sel.size();
  std::vector<int> sel_off(nt + 1, 0);
  for (int t = 0; t < nt; ++t) sel_off[t + 1] = sel_off[t] + sel[t];
  nl.N = N; nl.S = sel_off[nt];
  nl.j.assign((size_t)N * nl.S, -1); nl.img.assign((size_t)N * nl.S, 0);
  nl.count.assign((size_t)N * nt, 0);
  int nmax[3];
  // |n_a| <= ceil(rcut / w_a) for positions wrapped into the cell; one more for a triclinic
  // cell, whose wrapped fractional coordinates may round just outside [0, 1)
  for (int a = 0; a < 3; ++a) nmax[a] = (int)std::ceil(rcut / B.w[a]) + (B.tri ? 1 : 0);
  double rc2 = rcut * rcut;
  int ovf = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : ovf)
  for (int i = 0; i < N; ++i) {
    std::vector<Cand> c;
    for (int j = 0; j < N; ++j)
      for (int nx = -nmax[0]; nx <= nmax[0]; ++nx)
        for (int ny = -nmax[1]; ny <= nmax[1]; ++ny)
          for (int nz = -nmax[2]; nz <= nmax[2]; ++nz) {
            if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
            int n[3] = {nx, ny, nz};
            double r2 = dist2(&xw[3 * i], &xw[3 * j], n, B);
            if (r2 < rc2) c.push_back({types[j], j, pack_img(nx, ny, nz), r2});
          }
    std::sort(c.begin(), c.end(), cand_less);
    if (nearest) keep_nearest(c, sel, nt);
    emit(nl, i, c, sel, sel_off, nt);
    for (int t = 0; t < nt; ++t) if (nl.count[(size_t)i * nt + t] > sel[t]) ovf = 1;
  }
  nl.overflow = ovf != 0;
}

// Cell list: nc = max(1, floor(w / rcut)) cells per axis (w the perpendicular width; L for an
// orthorhombic box, with cells of edge L/nc), stencil of +-m cells with m = ceil(rcut / (w/nc))
// (one more for a triclinic cell, binned by fractional coordinate); virtual cell c + o maps to
// cell (c+o) mod nc with image shift floor((c+o) / nc).  Each (j, n) is visited at most once.
void nlist_cell(int N, const double* xw, const int* types, const Box& B, double rcut,
                const std::vector<int>& sel, NList& nl, bool nearest = false) {
  int nt = (int)sel.size();
  std::vector<int> sel_off(nt + 1, 0);
  for (int t = 0; t < nt; ++t) sel_off[t + 1] = sel_off[t] + sel[t];
  nl.N = N; nl.S = sel_off[nt];
  nl.j.assign((size_t)N * nl.S, -1); nl.img.assign((size_t)N * nl.S, 0);
  nl.count.assign((size_t)N * nt, 0);
  int nc[3], m[3];
  double edge[3];
  for (int a = 0; a < 3; ++a) {
    nc[a] = std::max(1, (int)std::floor(B.w[a] / rcut));
    edge[a] = B.w[a] / nc[a];
    m[a] = (int)std::ceil(rcut / edge[a]) + (B.tri ? 1 : 0);
  }
  size_t ncell = (size_t)nc[0] * nc[1] * nc[2];
  std::vector<int> cell_of(N);
  std::vector<std::vector<int>> members(ncell);
  for (int i = 0; i < N; ++i) {
    int c[3];
    double sf[3];
    if (B.tri) frac(B, &xw[3 * i], sf);
    for (int a = 0; a < 3; ++a) {
      c[a] = B.tri ? (int)std::floor(sf[a] * nc[a]) : (int)std::floor(xw[3 * i + a] / edge[a]);
      c[a] = std::min(std::max(c[a], 0), nc[a] - 1);
    }
    size_t id = ((size_t)c[0] * nc[1] + c[1]) * nc[2] + c[2];
    cell_of[i] = (int)id;
    members[id].push_back(i);
  }
  double rc2 = rcut * rcut;
  int ovf = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : ovf)
  for (int i = 0; i < N; ++i) {
    int ci[3];
    size_t id = cell_of[i];
    ci[2] = (int)(id % nc[2]); ci[1] = (int)((id / nc[2]) % nc[1]); ci[0] = (int)(id / ((size_t)nc[1] * nc[2]));
    std::vector<Cand> c;
    for (int ox = -m[0]; ox <= m[0]; ++ox)
      for (int oy = -m[1]; oy <= m[1]; ++oy)
        for (int oz = -m[2]; oz <= m[2]; ++oz) {
          int v[3] = {ci[0] + ox, ci[1] + oy, ci[2] + oz}, cc[3], n[3];
          for (int a = 0; a < 3; ++a) {
            int q = v[a];
            int fl = (q >= 0) ? q / nc[a] : -((-q + nc[a] - 1) / nc[a]);
            n[a] = fl;
            cc[a] = q - fl * nc[a];
          }
          size_t cid = ((size_t)cc[0] * nc[1] + cc[1]) * nc[2] + cc[2];
          for (int j : members[cid]) {
            if (j == i && n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
            double r2 = dist2(&xw[3 * i], &xw[3 * j], n, B);
            if (r2 < rc2) c.push_back({types[j], j, pack_img(n[0], n[1], n[2]), r2});
          }
        }
    std::sort(c.begin(), c.end(), cand_less);
    if (nearest) keep_nearest(c, sel, nt);
    emit(nl, i, c, sel, sel_off, nt);
    for (int t = 0; t < nt; ++t) if (nl.count[(size_t)i * nt + t] > sel[t]) ovf = 1;
  }
  nl.overflow = ovf != 0;
}

// Keep, in order, the entries of a (rcut + skin) list whose current distance is
// below rcut.  Positions are those of the current step (not re-wrapped).  With `nearest`, a type
// with more than sel_t such entries keeps its sel_t nearest (r^2, then j, then image).
void nlist_filter(const NList& big, int N, const double* x, const Box& B, double rcut,
                  const std::vector<int>& sel, const std::vector<int>& big_sel, NList& nl,
                  bool nearest = false) {
  int nt = (int)sel.size();
  std::vector<int> sel_off(nt + 1, 0), bsel_off(nt + 1, 0);
  for (int t = 0; t < nt; ++t) { sel_off[t + 1] = sel_off[t] + sel[t]; bsel_off[t + 1] = bsel_off[t] + big_sel[t]; }
  nl.N = N; nl.S = sel_off[nt];
  nl.j.assign((size_t)N * nl.S, -1); nl.img.assign((size_t)N * nl.S, 0);
  nl.count.assign((size_t)N * nt, 0);
  double rc2 = rcut * rcut;
  int ovf = 0;
#pragma omp parallel for schedule(static) reduction(| : ovf)
  for (int i = 0; i < N; ++i) {
    for (int t = 0; t < nt; ++t) {
      std::vector<Cand> c;
      for (int q = 0; q < big_sel[t]; ++q) {
        size_t e = (size_t)i * big.S + bsel_off[t] + q;
        int j = big.j[e];
        if (j < 0) break;
        int n[3];
        unpack_img(big.img[e], n[0], n[1], n[2]);
        double r2 = dist2(&x[3 * i], &x[3 * j], n, B);
        if (r2 < rc2) c.push_back({t, j, big.img[e], r2});
      }
      if (nearest && (int)c.size() > sel[t]) {
        std::vector<Cand> byr = c;
        std::sort(byr.begin(), byr.end(), cand_nearer);
        const Cand& last = byr[sel[t] - 1];
        std::vector<Cand> kept;
        for (const Cand& y : c)
          if (!cand_nearer(last, y)) kept.push_back(y);  // y ranks at or before the sel_t-th
        c.swap(kept);
      }
      int k = 0;
      for (const Cand& y : c) {
        if (k < sel[t]) { nl.j[(size_t)i * nl.S + sel_off[t] + k] = y.j; nl.img[(size_t)i * nl.S + sel_off[t] + k] = y.img; }
        ++k;
      }
      nl.count[(size_t)i * nt + t] = k;
      if (k > sel[t]) ovf = 1;
    }
  }
  nl.overflow = ovf != 0;
}

// ---------------------------------------------------------------- switch
// Quintic (C2) switch: u = (r - rs)/(rc - rs), sw = u^3(-6u^2 + 15u - 10) + 1 on
// [rs, rc); 1 below rs; 0 at and beyond rc.  Cosine alternative:
// sw = (cos(pi u) + 1)/2 on [rs, rc).
template <class T>
T switch_fn(T r, double rs, double rc, int kind) {
  if (val(r) < rs) return T(1.0);
  if (val(r) >= rc) return T(0.0);
  T u = (r - T(rs)) / T(rc - rs);
  if (kind == 1) return T(0.5) * cos(T(kPi) * u) + T(0.5);
  T u2 = u * u;
  T u3 = u2 * u;
  return u3 * (T(-6.0) * u2 + T(15.0) * u - T(10.0)) + T(1.0);
}

// ---------------------------------------------------------------- networks
// Embedding net forward for scalar input x; keeps the tanh outputs of each layer.
template <class T>
void emb_forward(const T* p, const Sizes& s, T x, std::vector<T>& h1, std::vector<T>& t2,
                 std::vector<T>& h2, std::vector<T>& t3, std::vector<T>& g) {
  const T* W1 = p;           const T* b1 = W1 + s.n1;
  const T* W2 = b1 + s.n1;   const T* b2 = W2 + (size_t)s.n1 * s.n2;
  const T* W3 = b2 + s.n2;   const T* b3 = W3 + (size_t)s.n2 * s.n3;
  h1.resize(s.n1); t2.resize(s.n2); h2.resize(s.n2); t3.resize(s.n3); g.resize(s.n3);
  for (int k = 0; k < s.n1; ++k) h1[k] = tanh(x * W1[k] + b1[k]);
  for (int m = 0; m < s.n2; ++m) {
    T z = b2[m];
    for (int k = 0; k < s.n1; ++k) z += h1[k] * W2[(size_t)k * s.n2 + m];
    t2[m] = tanh(z);
    T res = T(0.0);
    if (s.n2 == s.n1) res = h1[m];
    else if (s.n2 == 2 * s.n1) res = h1[m % s.n1];
    h2[m] = res + t2[m];
  }
  for (int a = 0; a < s.n3; ++a) {
    T z = b3[a];
    for (int m = 0; m < s.n2; ++m) z += h2[m] * W3[(size_t)m * s.n3 + a];
    t3[a] = tanh(z);
    T res = T(0.0);
    if (s.n3 == s.n2) res = h2[a];
    else if (s.n3 == 2 * s.n2) res = h2[a % s.n2];
    g[a] = res + t3[a];
  }
}

// Reverse of emb_forward: dG -> d(input).
template <class T>
T emb_backward(const T* p, const Sizes& s, const std::vector<T>& h1, const std::vector<T>& t2,
               const std::vector<T>& t3, const std::vector<T>& dg) {
  const T* W1 = p;           const T* b1 = W1 + s.n1;
  const T* W2 = b1 + s.n1;   const T* b2 = W2 + (size_t)s.n1 * s.n2;
  const T* W3 = b2 + s.n2;
  (void)b2;
  std::vector<T> dh2(s.n2, T(0.0)), dh1(s.n1, T(0.0));
  for (int a = 0; a < s.n3; ++a) {
    T dz = dg[a] * (T(1.0) - t3[a] * t3[a]);
    for (int m = 0; m < s.n2; ++m) dh2[m] += dz * W3[(size_t)m * s.n3 + a];
    if (s.n3 == s.n2) dh2[a] += dg[a];
    else if (s.n3 == 2 * s.n2) dh2[a % s.n2] += dg[a];
  }
  for (int m = 0; m < s.n2; ++m) {
    T dz = dh2[m] * (T(1.0) - t2[m] * t2[m]);
    for (int k = 0; k < s.n1; ++k) dh1[k] += dz * W2[(size_t)k * s.n2 + m];
    if (s.n2 == s.n1) dh1[m] += dh2[m];
    else if (s.n2 == 2 * s.n1) dh1[m % s.n1] += dh2[m];
  }
  T dx = T(0.0);
  for (int k = 0; k < s.n1; ++k) dx += dh1[k] * (T(1.0) - h1[k] * h1[k]) * W1[k];
  return dx;
}

// Tabulated embedding of pair `pair` at input x: G[a] and dG[a]/dx from the quintic of the
// interval holding x (inputs below the first node or above the last use the edge interval's
// polynomial).
template <class T, class M>
void tab_eval(const M& m, int pair, T x, std::vector<T>& g, std::vector<T>* dg) {
  const int n3 = m.sz.n3;
  g.resize(n3);
  if (dg) dg->resize(n3);
  int i = (int)std::floor((val(x) - m.tab_x0) / m.tab_h);
  i = std::min(std::max(i, 0), m.tab_n - 1);
  const T u = (x - T(m.tab_x0 + i * m.tab_h)) * T(1.0 / m.tab_h);
  for (int a = 0; a < n3; ++a) {
    const double* c = &m.tab[(((size_t)pair * m.tab_n + i) * n3 + a) * 6];
    g[a] = T(c[0]) + u * (T(c[1]) + u * (T(c[2]) + u * (T(c[3]) + u * (T(c[4]) + u * T(c[5])))));
    if (dg)
      (*dg)[a] = (T(c[1]) + u * (T(2.0 * c[2]) + u * (T(3.0 * c[3]) + u * (T(4.0 * c[4]) + u * T(5.0 * c[5]))))) *
                 T(1.0 / m.tab_h);
  }
}

// Build the table: at every node x_i = x0 + i h the embedding net's value, first and second
// derivative (second-order jets through emb_forward); on each interval the quintic in u with
// those six end conditions (value, h * first, h^2 * second derivative at u = 0 and u = 1).
void build_table(Model<double>& m, double x0, double x1, int n) {
  const Sizes& s = m.sz;
  const int nt = m.ntypes, n3 = s.n3;
  m.tab_n = n; m.tab_x0 = x0; m.tab_h = (x1 - x0) / n;
  const double h = m.tab_h;
  m.tab.assign((size_t)nt * nt * n * n3 * 6, 0.0);
  std::vector<Jet2> w(m.emb_size());
  for (int pair = 0; pair < nt * nt; ++pair) {
    for (size_t q = 0; q < w.size(); ++q) w[q] = Jet2(m.theta[m.emb_off[pair] + q]);
    std::vector<double> f((size_t)(n + 1) * n3), f1(f.size()), f2(f.size());
#pragma omp parallel for schedule(static)
    for (int i = 0; i <= n; ++i) {
      std::vector<Jet2> a1, a2, a3, a4, g;
      emb_forward(w.data(), s, Jet2(x0 + i * h, 1.0, 0.0), a1, a2, a3, a4, g);
      for (int a = 0; a < n3; ++a) {
        f[(size_t)i * n3 + a] = g[a].v;
        f1[(size_t)i * n3 + a] = g[a].d;
        f2[(size_t)i * n3 + a] = g[a].dd;
      }
    }
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < n3; ++a) {
        const size_t l = (size_t)i * n3 + a, r = l + n3;
        const double c0 = f[l], c1 = h * f1[l], c2 = 0.5 * h * h * f2[l];
        const double A = f[r] - (c0 + c1 + c2), B = h * f1[r] - (c1 + 2.0 * c2), C = h * h * f2[r] - 2.0 * c2;
        double* c = &m.tab[(((size_t)pair * n + i) * n3 + a) * 6];
        c[0] = c0; c[1] = c1; c[2] = c2;
        c[3] = 10.0 * A - 4.0 * B + 0.5 * C;
        c[4] = -15.0 * A + 7.0 * B - C;
        c[5] = 6.0 * A - 3.0 * B + 0.5 * C;
      }
  }
}

// Fitting net forward + reverse: returns E_i (without e_bias) and dE/dD.
template <class T>
T fit_forward_backward(const T* p, const Sizes& s, const std::vector<T>& D, std::vector<T>* dD) {
  const int K = s.n3 * s.m2;
  const T* W1 = p;          const T* b1 = W1 + (size_t)K * s.f1;
  const T* W2 = b1 + s.f1;  const T* b2 = W2 + (size_t)s.f1 * s.f2;
  const T* W3 = b2 + s.f2;  const T* b3 = W3 + (size_t)s.f2 * s.f3;
  const T* w4 = b3 + s.f3;  const T* b4 = w4 + s.f3;
  std::vector<T> h1(s.f1), t2(s.f2), h2(s.f2), t3(s.f3), h3(s.f3);
  for (int o = 0; o < s.f1; ++o) {
    T z = b1[o];
    for (int k = 0; k < K; ++k) z += D[k] * W1[(size_t)k * s.f1 + o];
    h1[o] = tanh(z);
  }
  for (int o = 0; o < s.f2; ++o) {
    T z = b2[o];
    for (int k = 0; k < s.f1; ++k) z += h1[k] * W2[(size_t)k * s.f2 + o];
    t2[o] = tanh(z);
    h2[o] = (s.f2 == s.f1 ? h1[o] : T(0.0)) + t2[o];
  }
  for (int o = 0; o < s.f3; ++o) {
    T z = b3[o];
    for (int k = 0; k < s.f2; ++k) z += h2[k] * W3[(size_t)k * s.f3 + o];
    t3[o] = tanh(z);
    h3[o] = (s.f3 == s.f2 ? h2[o] : T(0.0)) + t3[o];
  }
  T E = b4[0];
  for (int o = 0; o < s.f3; ++o) E += h3[o] * w4[o];
  if (!dD) return E;
  std::vector<T> dh2(s.f2, T(0.0)), dh1(s.f1, T(0.0));
  for (int o = 0; o < s.f3; ++o) {
    T dh3 = w4[o];
    T dz = dh3 * (T(1.0) - t3[o] * t3[o]);
    for (int k = 0; k < s.f2; ++k) dh2[k] += dz * W3[(size_t)k * s.f3 + o];
    if (s.f3 == s.f2) dh2[o] += dh3;
  }
  for (int o = 0; o < s.f2; ++o) {
    T dz = dh2[o] * (T(1.0) - t2[o] * t2[o]);
    for (int k = 0; k < s.f1; ++k) dh1[k] += dz * W2[(size_t)k * s.f2 + o];
    if (s.f2 == s.f1) dh1[o] += dh2[o];
  }
  dD->assign(K, T(0.0));
  for (int o = 0; o < s.f1; ++o) {
    T dz = dh1[o] * (T(1.0) - h1[o] * h1[o]);
    for (int k = 0; k < K; ++k) (*dD)[k] += dz * W1[(size_t)k * s.f1 + o];
  }
  return E;
}

// ---------------------------------------------------------------- one evaluation
struct Inter {            // optional per-atom intermediates
  double* T = nullptr;    // [N][4][n3]
  double* D = nullptr;    // [N][n3*m2]
  double* dD = nullptr;   // [N][n3*m2]
  double* W = nullptr;    // [N][9] per-atom virial: -sum over atom i's neighbours of g (x) d
};

// Energy, forces and virial for all atoms whose centre_mask is set (all if null).
// x may be Dual (directional derivatives); positions used for the geometry are
// x itself, the neighbour list nl is fixed.
template <class T>
void evaluate(const Model<T>& m, int N, const T* x, const int* types, const Box& B,
              const NList& nl, const unsigned char* centre_mask, bool want_force, T* energy,
              T* atom_energy, T* force, T* virial, const Inter* inter) {
  const Sizes& s = m.sz;
  const int S = m.S, nt = m.ntypes, M2 = s.m2, n3 = s.n3;
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  std::vector<std::vector<T>> fbuf(nthreads), vbuf(nthreads, std::vector<T>(9, T(0.0)));
  std::vector<T> Ei(N, T(0.0));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    if (want_force) fbuf[tid].assign((size_t)N * 3, T(0.0));
    std::vector<T> R((size_t)S * 4), dvec((size_t)S * 3), rr(S);
    std::vector<std::vector<T>> h1(S), t2(S), h2(S), t3(S), G(S);
    std::vector<T> Tm((size_t)4 * n3), Dm((size_t)n3 * M2), dD, dT((size_t)4 * n3);
    std::vector<T> ph1, pt2, ph2, pt3, Gp;  // embedding of a padded slot
#pragma omp for schedule(dynamic, 4)
    for (int i = 0; i < N; ++i) {
      if (centre_mask && !centre_mask[i]) continue;
      const int ti = types[i];
      // environment matrix rows
      for (int k = 0; k < S; ++k) {
        int j = nl.j[(size_t)i * nl.S + k];
        if (j < 0) continue;
        int n[3];
        unpack_img(nl.img[(size_t)i * nl.S + k], n[0], n[1], n[2]);
        T d[3];
        for (int a = 0; a < 3; ++a) d[a] = (x[3 * j + a] + T(shift(B, n, a))) - x[3 * i + a];
        T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        T sw = switch_fn(r, m.rs, m.rc, m.switch_kind);
        T sv = sw / r;
        T row[4] = {sv, sv * d[0] / r, sv * d[1] / r, sv * d[2] / r};
        for (int c = 0; c < 4; ++c) R[(size_t)k * 4 + c] = (row[c] - T(m.davg[ti * 4 + c])) / T(m.dstd[ti * 4 + c]);
        for (int a = 0; a < 3; ++a) dvec[(size_t)k * 3 + a] = d[a];
        rr[k] = r;
        const int tj = types[j];
        if (m.tab_n > 0) tab_eval(m, ti * nt + tj, R[(size_t)k * 4], G[k], &t3[k]);  // t3: dG/dx
        else emb_forward(&m.theta[m.emb_off[ti * nt + tj]], s, R[(size_t)k * 4], h1[k], t2[k], h2[k], t3[k], G[k]);
      }
      // T = (1/S) R^T G over all S slots.  A padded slot is the row of an absent
      // neighbour, R_tilde = 0, normalised like every row: R_hat = -davg/dstd, with
      // G from the net of (ti, the slot's neighbour type).  It equals the row of a
      // neighbour sitting exactly at r_c (s = 0), so E stays continuous when a
      // neighbour crosses the cutoff.  Its G is the same for every padded slot of a
      // type segment and is computed once per atom and segment.
      for (size_t q = 0; q < Tm.size(); ++q) Tm[q] = T(0.0);
      for (int tj = 0; tj < nt; ++tj) {
        bool have_pad = false;
        T Rp[4];
        for (int c = 0; c < 4; ++c) Rp[c] = (T(0.0) - T(m.davg[ti * 4 + c])) / T(m.dstd[ti * 4 + c]);
        for (int k = m.sel_off[tj]; k < m.sel_off[tj + 1]; ++k) {
          const bool pad = nl.j[(size_t)i * nl.S + k] < 0;
          if (pad && !have_pad) {
            if (m.tab_n > 0) tab_eval(m, ti * nt + tj, Rp[0], Gp, (std::vector<T>*)nullptr);
            else emb_forward(&m.theta[m.emb_off[ti * nt + tj]], s, Rp[0], ph1, pt2, ph2, pt3, Gp);
            have_pad = true;
          }
          const T* Rk = pad ? Rp : &R[(size_t)k * 4];
          const std::vector<T>& Gk = pad ? Gp : G[k];
          for (int c = 0; c < 4; ++c)
            for (int a = 0; a < n3; ++a) Tm[(size_t)c * n3 + a] += Rk[c] * Gk[a];
        }
      }
      for (size_t q = 0; q < Tm.size(); ++q) Tm[q] = Tm[q] / T((double)S);
      // D = T^T T[:, :M2], flattened a*M2 + b
      for (int a = 0; a < n3; ++a)
        for (int b = 0; b < M2; ++b) {
          T acc = T(0.0);
          for (int c = 0; c < 4; ++c) acc += Tm[(size_t)c * n3 + a] * Tm[(size_t)c * n3 + b];
          Dm[(size_t)a * M2 + b] = acc;
        }
      T e = fit_forward_backward(&m.theta[m.fit_off[ti]], s, Dm, want_force ? &dD : nullptr);
      e += m.theta[m.ebias_off + ti];
      Ei[i] = e;
      if (inter && inter->T) for (size_t q = 0; q < Tm.size(); ++q) inter->T[(size_t)i * 4 * n3 + q] = val(Tm[q]);
      if (inter && inter->D) for (size_t q = 0; q < Dm.size(); ++q) inter->D[(size_t)i * n3 * M2 + q] = val(Dm[q]);
      if (!want_force) continue;
      if (inter && inter->dD) for (size_t q = 0; q < dD.size(); ++q) inter->dD[(size_t)i * n3 * M2 + q] = val(dD[q]);
      // dT[c][a] = sum_b dD[a][b] T[c][b] + [a < M2] sum_a' dD[a'][a] T[c][a']
      for (int c = 0; c < 4; ++c)
        for (int a = 0; a < n3; ++a) {
          T acc = T(0.0);
          for (int b = 0; b < M2; ++b) acc += dD[(size_t)a * M2 + b] * Tm[(size_t)c * n3 + b];
          if (a < M2)
            for (int a2 = 0; a2 < n3; ++a2) acc += dD[(size_t)a2 * M2 + a] * Tm[(size_t)c * n3 + a2];
          dT[(size_t)c * n3 + a] = acc;
        }
      for (int k = 0; k < S; ++k) {
        int j = nl.j[(size_t)i * nl.S + k];
        if (j < 0) continue;
        const int tj = types[j];
        // dR_hat[c] = (1/S) sum_a dT[c][a] G[a];  dG[a] = (1/S) sum_c R_hat[c] dT[c][a]
        T dR[4];
        for (int c = 0; c < 4; ++c) {
          T acc = T(0.0);
          for (int a = 0; a < n3; ++a) acc += dT[(size_t)c * n3 + a] * G[k][a];
          dR[c] = acc / T((double)S);
        }
        std::vector<T> dG(n3);
        for (int a = 0; a < n3; ++a) {
          T acc = T(0.0);
          for (int c = 0; c < 4; ++c) acc += R[(size_t)k * 4 + c] * dT[(size_t)c * n3 + a];
          dG[a] = acc / T((double)S);
        }
        if (m.tab_n > 0) {
          for (int a = 0; a < n3; ++a) dR[0] += dG[a] * t3[k][a];
        } else {
          dR[0] += emb_backward(&m.theta[m.emb_off[ti * nt + tj]], s, h1[k], t2[k], t3[k], dG);
        }
        // undo normalisation, then the analytic Jacobian of (s, s d/r) w.r.t. d
        for (int c = 0; c < 4; ++c) dR[c] = dR[c] / T(m.dstd[ti * 4 + c]);
        T r = rr[k];
        const T* d = &dvec[(size_t)k * 3];
        // sw'(r)
        T sw, dsw;
        if (val(r) < m.rs) { sw = T(1.0); dsw = T(0.0); }
        else if (val(r) >= m.rc) { sw = T(0.0); dsw = T(0.0); }
        else {
          T w = T(m.rc - m.rs);
          T u = (r - T(m.rs)) / w;
          if (m.switch_kind == 1) {
            sw = T(0.5) * cos(T(kPi) * u) + T(0.5);
            dsw = T(-0.5 * kPi) * sin(T(kPi) * u) / w;
          } else {
            T u2 = u * u;
            sw = u2 * u * (T(-6.0) * u2 + T(15.0) * u - T(10.0)) + T(1.0);
            dsw = T(-30.0) * u2 * (u - T(1.0)) * (u - T(1.0)) / w;
          }
        }
        // s = sw/r, ds/dr = sw'/r - sw/r^2 ; q = sw/r^2, dq/dr = sw'/r^2 - 2 sw/r^3
        T ds = dsw / r - sw / (r * r);
        T qv = sw / (r * r);
        T dq = dsw / (r * r) - T(2.0) * sw / (r * r * r);
        T proj = dR[1] * d[0] + dR[2] * d[1] + dR[3] * d[2];
        T common = (dR[0] * ds + dq * proj) / r;
        T g[3];
        for (int a = 0; a < 3; ++a) g[a] = common * d[a] + qv * dR[1 + a];
        std::vector<T>& F = fbuf[tid];
        for (int a = 0; a < 3; ++a) { F[3 * i + a] += g[a]; F[3 * j + a] -= g[a]; }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            vbuf[tid][a * 3 + b] -= g[a] * d[b];
            if (inter && inter->W) inter->W[(size_t)i * 9 + a * 3 + b] -= val(g[a] * d[b]);
          }
      }
    }
  }
  T E = T(0.0);
  for (int i = 0; i < N; ++i) E += Ei[i];
  if (energy) *energy = E;
  if (atom_energy) for (int i = 0; i < N; ++i) atom_energy[i] = Ei[i];
  if (want_force) {
    if (force) {
      for (size_t q = 0; q < (size_t)N * 3; ++q) force[q] = T(0.0);
      for (int t = 0; t < nthreads; ++t)
        if (!fbuf[t].empty()) for (size_t q = 0; q < (size_t)N * 3; ++q) force[q] += fbuf[t][q];
    }
    if (virial) {
      for (int q = 0; q < 9; ++q) virial[q] = T(0.0);
      for (int t = 0; t < nthreads; ++t) for (int q = 0; q < 9; ++q) virial[q] += vbuf[t][q];
    }
  }
}

// Orthorhombic: wrap1 per axis.  Triclinic: t = floor(x Hinv) (fractional coordinates, fixed
// order) and w = x - t H, each component ((t0 H0c + t1 H1c) + t2 H2c) subtracted from x_c.
void wrap_all(int N, const double* x, const Box& B, std::vector<double>& xw) {
  xw.resize((size_t)N * 3);
  for (int i = 0; i < N; ++i) {
    if (!B.tri) {
      for (int a = 0; a < 3; ++a) xw[3 * i + a] = wrap1(x[3 * i + a], B.L[a]);
      continue;
    }
    double sf[3];
    frac(B, &x[3 * i], sf);
    int t[3] = {(int)std::floor(sf[0]), (int)std::floor(sf[1]), (int)std::floor(sf[2])};
    for (int c = 0; c < 3; ++c) xw[3 * i + c] = x[3 * i + c] - shift(B, t, c);
  }
}

// Box from the caller's [9] (rows a, b, c).  Any right-handed cell of positive volume; its
// inverse is the adjugate over the determinant, each cofactor a difference of two products.
bool box_geom(const double* box, Box& B) {
  for (int q = 0; q < 9; ++q) { if (!std::isfinite(box[q])) return false; B.H[q] = box[q]; }
  B.tri = false;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b && box[a * 3 + b] != 0.0) B.tri = true;
  const double* h = B.H;
  double cof[9];  // cof[3r + c] = cofactor of entry (r, c)
  cof[0] = h[4] * h[8] - h[5] * h[7];
  cof[1] = h[5] * h[6] - h[3] * h[8];
  cof[2] = h[3] * h[7] - h[4] * h[6];
  cof[3] = h[2] * h[7] - h[1] * h[8];
  cof[4] = h[0] * h[8] - h[2] * h[6];
  cof[5] = h[1] * h[6] - h[0] * h[7];
  cof[6] = h[1] * h[5] - h[2] * h[4];
  cof[7] = h[2] * h[3] - h[0] * h[5];
  cof[8] = h[0] * h[4] - h[1] * h[3];
  const double det = (h[0] * cof[0] + h[1] * cof[1]) + h[2] * cof[2];
  if (!(det > 0.0)) return false;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) B.Hinv[3 * r + c] = cof[3 * c + r] / det;  // inverse = adj^T / det
  // |b x c| = norm of cofactor row 0, etc.
  for (int a = 0; a < 3; ++a) {
    const double* k = cof + 3 * a;
    B.w[a] = det / std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    B.L[a] = h[4 * a];
  }
  if (!B.tri)
    for (int a = 0; a < 3; ++a) { B.w[a] = B.L[a]; if (!(B.L[a] > 0.0)) return false; }
  return true;
}

}  // namespace

// ================================================================ C interface
extern "C" {

// Status codes: 0 ok, 1 bad argument, 4 unsupported box, 5 neighbour overflow, 9 bad weights.

void* oracle_model_load(const void* blob, size_t nbytes) {
  auto* m = new Model<double>();
  if (!load_model(blob, nbytes, *m)) { delete m; return nullptr; }
  return m;
}

void oracle_model_free(void* h) { delete static_cast<Model<double>*>(h); }

// Neighbour overflow policy: 0 = a type with more than sel_t neighbours is an error (status 5),
// 1 = nearest-first truncation (keep the sel_t nearest by r^2, then j, then image).
int oracle_set_truncation(void* h, int nearest) {
  static_cast<Model<double>*>(h)->nearest = nearest != 0;
  return 0;
}

long long oracle_model_ntheta(const void* h) { return (long long)static_cast<const Model<double>*>(h)->ntheta; }
int oracle_model_ntypes(const void* h) { return static_cast<const Model<double>*>(h)->ntypes; }
int oracle_model_S(const void* h) { return static_cast<const Model<double>*>(h)->S; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Wrap positions into the box (same rule as the neighbour list uses).
int oracle_wrap(int N, const double* x, const double* box, double* xw) {
  Box B;
  if (!box_geom(box, B)) return 4;
  std::vector<double> w;
  wrap_all(N, x, B, w);
  std::memcpy(xw, w.data(), sizeof(double) * 3 * N);
  return 0;
}

// Canonical neighbour list of the wrapped positions within `rcut` (or the model's
// r_c when rcut <= 0).  method 0 = brute force, 1 = cell list.  nlist/images are
// [N][S] padded with -1 / 0; counts [N][nt] are the true per-type counts.
int oracle_nlist(const void* h, int N, const double* x, const int* types, const double* box,
                 double rcut, const int* sel_override, int method, int* nlist, int* images, int* counts) {
  const Model<double>& m = *static_cast<const Model<double>*>(h);
  Box B;
  if (!box_geom(box, B)) return 4;
  std::vector<double> xw;
  wrap_all(N, x, B, xw);
  std::vector<int> sel = m.sel;
  if (sel_override) for (int t = 0; t < m.ntypes; ++t) sel[t] = sel_override[t];
  NList nl;
  double rc = rcut > 0 ? rcut : m.rc;
  if (method == 0) nlist_brute(N, xw.data(), types, B, rc, sel, nl, m.nearest);
  else nlist_cell(N, xw.data(), types, B, rc, sel, nl, m.nearest);
  if (nlist) std::memcpy(nlist, nl.j.data(), sizeof(int) * nl.j.size());
  if (images) std::memcpy(images, nl.img.data(), sizeof(int) * nl.img.size());
  if (counts) std::memcpy(counts, nl.count.data(), sizeof(int) * nl.count.size());
  return nl.overflow ? 5 : 0;
}

// Energy, per-atom energy, forces, virial of one periodic box (positions wrapped
// first).  centre_mask (nullable, [N]) restricts the sum over centres, so forces are
// exact only on atoms whose whole r_c neighbourhood is masked in.  Intermediates
// T/D/dD (nullable) are written per atom.
int oracle_compute(const void* h, int N, const double* x, const int* types, const double* box,
                   int method, const unsigned char* centre_mask, int want_force, double* energy,
                   double* atom_energy, double* force, double* virial, double* interT,
                   double* interD, double* interdD, double* atom_virial) {
  const Model<double>& m = *static_cast<const Model<double>*>(h);
  Box B;
  if (!box_geom(box, B)) return 4;
  std::vector<double> xw;
  wrap_all(N, x, B, xw);
  NList nl;
  if (method == 0) nlist_brute(N, xw.data(), types, B, m.rc, m.sel, nl, m.nearest);
  else nlist_cell(N, xw.data(), types, B, m.rc, m.sel, nl, m.nearest);
  if (nl.overflow) return 5;
  if (atom_virial) for (size_t q = 0; q < (size_t)N * 9; ++q) atom_virial[q] = 0.0;
  Inter in{interT, interD, interdD, atom_virial};
  evaluate<double>(m, N, xw.data(), types, B, nl, centre_mask, want_force != 0, energy, atom_energy,
                   force, virial, &in);
  return 0;
}

// Pair-distance histogram within r_max (<= any r): for every atom i and neighbour (j, n) at
// distance r < r_max (brute-force cell list, wrapped positions, r^2 in the fixed operation order),
// counts[(t_i * nt + t_j) * nbins + min(floor(r * nbins / r_max), nbins - 1)] += 1.
int oracle_rdf(const void* h, int N, const double* x, const int* types, const double* box, int nbins,
               double r_max, unsigned long long* counts) {
  const Model<double>& m = *static_cast<const Model<double>*>(h);
  Box B;
  if (!box_geom(box, B)) return 4;
  if (nbins < 1 || !(r_max > 0)) return 1;
  std::vector<double> xw;
  wrap_all(N, x, B, xw);
  const int nt = m.ntypes;
  std::vector<int> big(nt, N * 64);
  NList nl;
  nlist_cell(N, xw.data(), types, B, r_max, big, nl);
  for (size_t q = 0; q < (size_t)nt * nt * nbins; ++q) counts[q] = 0;
  const double inv = nbins / r_max;
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < nl.S; ++k) {
      const int j = nl.j[(size_t)i * nl.S + k];
      if (j < 0) continue;
      int n[3];
      unpack_img(nl.img[(size_t)i * nl.S + k], n[0], n[1], n[2]);
      const double r = std::sqrt(dist2(&xw[3 * i], &xw[3 * j], n, B));
      const int b = std::min((int)std::floor(r * inv), nbins - 1);
      counts[((size_t)types[i] * nt + types[j]) * nbins + b] += 1;
    }
  return 0;
}

// Tabulate every embedding net of the model (compressed model): n uniform intervals on
// [x0, x1] (n = 0 goes back to the networks).  Returns 1 for bad arguments.
int oracle_tabulate(void* h, double x0, double x1, int n) {
  Model<double>& m = *static_cast<Model<double>*>(h);
  if (n < 0 || (n > 0 && !(x1 > x0))) return 1;
  if (n == 0) { m.tab_n = 0; m.tab.clear(); return 0; }
  build_table(m, x0, x1, n);
  return 0;
}

// The embedding output of pair (ti, tj) at nx inputs x: G [nx][n3] and its first and second
// derivatives, from the network (second-order jets, tabulated = 0) or from the table
// (tabulated = 1; second derivative of the quintic).
int oracle_emb_eval(const void* h, int pair, int nx, const double* x, int tabulated, double* g, double* g1,
                    double* g2) {
  const Model<double>& m = *static_cast<const Model<double>*>(h);
  const int n3 = m.sz.n3;
  if (pair < 0 || pair >= m.ntypes * m.ntypes || (tabulated && m.tab_n == 0)) return 1;
  std::vector<Jet2> w(m.emb_size());
  for (size_t q = 0; q < w.size(); ++q) w[q] = Jet2(m.theta[m.emb_off[pair] + q]);
  for (int k = 0; k < nx; ++k) {
    if (tabulated) {
      std::vector<Jet2> gj;
      Model<Jet2> mj;  // the table in jet arithmetic: second derivative of the quintic
      mj.sz = m.sz; mj.tab_n = m.tab_n; mj.tab_x0 = m.tab_x0; mj.tab_h = m.tab_h; mj.tab = m.tab;
      tab_eval(mj, pair, Jet2(x[k], 1.0, 0.0), gj, (std::vector<Jet2>*)nullptr);
      for (int a = 0; a < n3; ++a) {
        g[(size_t)k * n3 + a] = gj[a].v; g1[(size_t)k * n3 + a] = gj[a].d; g2[(size_t)k * n3 + a] = gj[a].dd;
      }
    } else {
      std::vector<Jet2> a1, a2, a3, a4, gj;
      emb_forward(w.data(), m.sz, Jet2(x[k], 1.0, 0.0), a1, a2, a3, a4, gj);
      for (int a = 0; a < n3; ++a) {
        g[(size_t)k * n3 + a] = gj[a].v; g1[(size_t)k * n3 + a] = gj[a].d; g2[(size_t)k * n3 + a] = gj[a].dd;
      }
    }
  }
  return 0;
}

// Environment statistics of one configuration, per centre type t (the input
// normalisation of the smooth descriptor, Section II-A): over every neighbour slot of
// every atom of type t -- S slots per atom, a padded slot counting as the zero row --
// of the un-normalised rows (s, s dx/r, s dy/r, s dz/r):
//   sums[5 t + 0] = number of slots, [1] = sum of s, [2] = sum of s^2,
//   [3] = sum of (s dx/r)^2 + (s dy/r)^2 + (s dz/r)^2, [4] = number of atoms.
int oracle_env_stats(const void* h, int N, const double* x, const int* types, const double* box, double* sums) {
  const Model<double>& m = *static_cast<const Model<double>*>(h);
  Box B;
  if (!box_geom(box, B)) return 4;
  std::vector<double> xw;
  wrap_all(N, x, B, xw);
  NList nl;
  nlist_cell(N, xw.data(), types, B, m.rc, m.sel, nl, m.nearest);
  if (nl.overflow) return 5;
  for (int q = 0; q < 5 * m.ntypes; ++q) sums[q] = 0.0;
  for (int i = 0; i < N; ++i) {
    double* o = sums + 5 * types[i];
    o[0] += m.S;
    o[4] += 1.0;
    for (int k = 0; k < m.S; ++k) {
      const int j = nl.j[(size_t)i * nl.S + k];
      if (j < 0) continue;  // the zero row adds nothing to the sums
      int n[3];
      unpack_img(nl.img[(size_t)i * nl.S + k], n[0], n[1], n[2]);
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = (xw[3 * j + a] + shift(B, n, a)) - xw[3 * i + a];
      const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double sv = switch_fn(r, m.rs, m.rc, m.switch_kind) / r;
      o[1] += sv;
      o[2] += sv * sv;
      for (int a = 0; a < 3; ++a) o[3] += (sv * d[a] / r) * (sv * d[a] / r);
    }
  }
  return 0;
}

// Directional derivative of E along displacement w ([N][3]) with dual numbers:
// out[0] = E, out[1] = sum_k w_k . dE/dx_k (exact up to rounding).
int oracle_dir_deriv(const void* h, int N, const double* x, const int* types, const double* box,
                     const double* w, double* out) {
  const Model<double>& md = *static_cast<const Model<double>*>(h);
  Box B;
  if (!box_geom(box, B)) return 4;
  std::vector<double> xw;
  wrap_all(N, x, B, xw);
  NList nl;
  nlist_cell(N, xw.data(), types, B, md.rc, md.sel, nl, md.nearest);
  if (nl.overflow) return 5;
  Model<Dual> m = cast_model<Dual>(md);
  std::vector<Dual> xd((size_t)N * 3);
  for (size_t q = 0; q < xd.size(); ++q) xd[q] = Dual(xw[q], w[q]);
  Dual E;
  evaluate<Dual>(m, N, xd.data(), types, B, nl, nullptr, false, &E, nullptr, nullptr, nullptr, nullptr);
  out[0] = E.v; out[1] = E.d;
  return 0;
}

// Parameter gradient of L = cE*(E - E0)^2 + cF*|F - F0|^2 for the chosen theta
// indices, by forward-mode dual numbers seeded on each theta_p in turn (E and F
// come out with exact tangents dE/dtheta_p, dF/dtheta_p).  Also returns
// dE/dtheta_p and the loss.  F0 is [N][3] in the caller's atom order.
int oracle_param_grad(const void* h, int N, const double* x, const int* types, const double* box,
                      double E0, const double* F0, double cE, double cF, int np, const long long* idx,
                      double* grad, double* dEdtheta, double* loss) {
  const Model<double>& md = *static_cast<const Model<double>*>(h);
  Box B;
  if (!box_geom(box, B)) return 4;
  std::vector<double> xw;
  wrap_all(N, x, B, xw);
  NList nl;
  nlist_cell(N, xw.data(), types, B, md.rc, md.sel, nl, md.nearest);
  if (nl.overflow) return 5;
  Model<Dual> m = cast_model<Dual>(md);
  std::vector<Dual> xd((size_t)N * 3), F((size_t)N * 3);
  for (size_t q = 0; q < xd.size(); ++q) xd[q] = Dual(xw[q]);
  for (int p = 0; p < np; ++p) {
    if (idx[p] < 0 || idx[p] >= (long long)m.ntheta) return 1;
    m.theta[idx[p]].d = 1.0;
    Dual E, vir[9];
    evaluate<Dual>(m, N, xd.data(), types, B, nl, nullptr, true, &E, nullptr, F.data(), vir, nullptr);
    m.theta[idx[p]].d = 0.0;
    double g = cE * 2.0 * (E.v - E0) * E.d;
    double lo = cE * (E.v - E0) * (E.v - E0);
    for (size_t q = 0; q < F.size(); ++q) {
      g += cF * 2.0 * (F[q].v - F0[q]) * F[q].d;
      lo += cF * (F[q].v - F0[q]) * (F[q].v - F0[q]);
    }
    grad[p] = g;
    if (dEdtheta) dEdtheta[p] = E.d;
    if (loss) *loss = lo;
  }
  return 0;
}

}  // extern "C"

namespace {

// Velocity-Verlet NVE loop shared by the model and the harmonic test force:
//   v += (dt/2) kappa F/m ; x += dt v ; [rebuild | displacement check] ;
//   F = force(x) ; v += (dt/2) kappa F/m
// kappa = 9.648533e-3 converts eV / (A amu) to A / fs^2.
template <class ForceFn, class RebuildFn, class CheckFn, class RecordFn>
int verlet_loop(int N, double* x, double* v, const std::vector<double>& mass, double dt, int nsteps,
                int rebuild_every, ForceFn force, RebuildFn rebuild, CheckFn check, RecordFn record,
                std::vector<double>& F) {
  const double kappa = 9.648533e-3;
  int st;
  for (int step = 0; step < nsteps; ++step) {
    for (int i = 0; i < N; ++i) {
      double a = 0.5 * dt * kappa / mass[i];
      for (int c = 0; c < 3; ++c) v[3 * i + c] += a * F[3 * i + c];
      for (int c = 0; c < 3; ++c) x[3 * i + c] += dt * v[3 * i + c];
    }
    if (rebuild_every > 0 && (step + 1) % rebuild_every == 0) {
      if ((st = rebuild())) return st;
    } else if ((st = check())) {
      return st;
    }
    double E = 0.0;
    if ((st = force(&E))) return st;
    for (int i = 0; i < N; ++i) {
      double a = 0.5 * dt * kappa / mass[i];
      for (int c = 0; c < 3; ++c) v[3 * i + c] += a * F[3 * i + c];
    }
    record(step + 1, E);
  }
  return 0;
}

double kinetic_energy(int N, const double* v, const std::vector<double>& mass) {
  double k = 0.0;
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) k += 0.5 * mass[i] * v[3 * i + a] * v[3 * i + a];
  return k / 9.648533e-3;
}

}  // namespace

extern "C" {

// Velocity-Verlet NVE with the model.  x, v [N][3] are updated in place (x ends
// wrapped at the last rebuild and drifted since).  masses per type in amu; dt in
// fs; the neighbour list (r_c + skin) is rebuilt at start and every
// `rebuild_every` steps.  pe/ke [nsteps + 1] receive potential and kinetic energy
// (eV) after each step (index 0 = initial state).  Returns 6 if an atom moved more
// than skin/2 since the last rebuild, 5 on neighbour overflow.
int oracle_md(const void* h, int N, double* x, double* v, const int* types, const double* box,
              const double* mass_by_type, double dt, int nsteps, int rebuild_every, double skin,
              double* pe, double* ke, double* force_out) {
  const Model<double>& m = *static_cast<const Model<double>*>(h);
  Box B;
  if (!box_geom(box, B)) return 4;
  const double rcs = m.rc + skin;
  std::vector<int> big_sel(m.ntypes);
  // Verlet-list capacity per type: generous multiple of sel scaled by volume.
  for (int t = 0; t < m.ntypes; ++t)
    big_sel[t] = (int)std::ceil(1.5 * m.sel[t] * std::pow(rcs / m.rc, 3.0)) + 32;
  std::vector<double> xw, xref((size_t)N * 3), F((size_t)N * 3), mass(N);
  for (int i = 0; i < N; ++i) mass[i] = mass_by_type[types[i]];
  NList big, nl;
  auto rebuild = [&]() -> int {
    wrap_all(N, x, B, xw);
    std::memcpy(x, xw.data(), sizeof(double) * 3 * N);
    std::memcpy(xref.data(), x, sizeof(double) * 3 * N);
    nlist_cell(N, x, types, B, rcs, big_sel, big);
    return big.overflow ? 5 : 0;
  };
  auto check = [&]() -> int {
    double lim = 0.25 * skin * skin;
    for (int i = 0; i < N; ++i) {
      double d2 = 0.0;
      for (int c = 0; c < 3; ++c) { double d = x[3 * i + c] - xref[3 * i + c]; d2 += d * d; }
      if (d2 > lim) return 6;
    }
    return 0;
  };
  auto force = [&](double* E) -> int {
    nlist_filter(big, N, x, B, m.rc, m.sel, big_sel, nl, m.nearest);
    if (nl.overflow) return 5;
    double vir[9];
    evaluate<double>(m, N, x, types, B, nl, nullptr, true, E, nullptr, F.data(), vir, nullptr);
    return 0;
  };
  auto record = [&](int k, double E) {
    if (pe) pe[k] = E;
    if (ke) ke[k] = kinetic_energy(N, v, mass);
  };
  int st = rebuild();
  if (st) return st;
  double E;
  if ((st = force(&E))) return st;
  record(0, E);
  st = verlet_loop(N, x, v, mass, dt, nsteps, rebuild_every, force, rebuild, check, record, F);
  if (force_out) std::memcpy(force_out, F.data(), sizeof(double) * 3 * N);
  return st;
}

// The same integrator driven by an isotropic harmonic tether F = -k x (eV/A^2),
// for checking the integrator against the closed-form oscillator.  traj
// [nsteps + 1][N][3] receives the positions after each step.
int oracle_md_harmonic(int N, double* x, double* v, const double* mass_per_atom, double k_spring,
                       double dt, int nsteps, double* traj) {
  std::vector<double> F((size_t)N * 3), mass(mass_per_atom, mass_per_atom + N);
  auto force = [&](double* E) -> int {
    double e = 0.0;
    for (size_t q = 0; q < F.size(); ++q) { F[q] = -k_spring * x[q]; e += 0.5 * k_spring * x[q] * x[q]; }
    *E = e;
    return 0;
  };
  auto none = [&]() -> int { return 0; };
  auto record = [&](int k, double) {
    if (traj) std::memcpy(traj + (size_t)k * 3 * N, x, sizeof(double) * 3 * N);
  };
  double E;
  force(&E);
  record(0, E);
  return verlet_loop(N, x, v, mass, dt, nsteps, 0, force, none, none, record, F);
}

}  // extern "C"
