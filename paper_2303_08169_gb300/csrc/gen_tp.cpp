// gen_tp.cpp - build-time generator of the channel-wise tensor-product code.
//
// Sec. 2.1 of the paper builds the energy from tensor products of irreducible
// representations.  The coupling tensors used here are the real-basis
// Clebsch-Gordan tensors of the natural-parity paths (l1, l2, l3), l1 + l2 + l3
// even, normalised to Frobenius norm 1 and signed so that coupling Y_l1(z)
// with Y_l2(z) gives a positive multiple of Y_l3(z).
//
// Method (independent of any other implementation in this repository): for
// even paths the real coupling tensor is proportional to the real Gaunt
// integral G[m1,m2,m3] = Int Y_l1m1 Y_l2m2 Y_l3m3 dOmega of the real spherical
// harmonics.  The integrand is a polynomial of degree <= 6 on the sphere, so a
// product rule with 8 Gauss-Legendre nodes in cos(theta) and 16 equispaced
// nodes in phi integrates it exactly.  G is then normalised and sign-fixed.
//
// Odd paths (l1 + l2 + l3 odd; full O(3), where they couple tensors of
// opposite parity): the Gaunt integral vanishes there, and the coupling is
// taken from another equivariant integral instead,
//   K[m1,m2,m3] = Int u . (grad R_l1m1 x grad R_l2m2) Y_l3m3 dOmega,
// with R_lm the harmonic homogeneous polynomials that equal Y_lm on the unit
// sphere.  Rotations act on u and on both gradients alike and the cross
// product of two rotated vectors is the rotated cross product, so K maps
// Y_l1 (x) Y_l2 equivariantly onto Y_l3; that map is unique up to a factor,
// so the normalised K is the real coupling tensor of the path.  Its integrand
// has degree <= 5, integrated exactly by the same rule.  Sign: the first
// nonzero entry in (m1, m2, m3) order is positive (no product of harmonics
// along one axis couples through an odd path: it is parity-odd).
//
// Output: a header with, per l_max in {0, 1, 2}, straight-line device
// function templates over the scalar type S (float, or the tangent numbers of
// the second-order adjoint)
//   tpL_fwd(V, G, T)          all paths            T[c-local layout below]
//   tpL_fwd_scalar(V, G, S)   l3 = 0 paths only
//   tpL_bwd(V, G, dT, dV, dG) adjoint of tpL_fwd (accumulates into dV, dG)
//   tpL_bwd_scalar(V, G, dS, dV, dG)
//   tpL_bwd_l3lt2 / tpL_bwd_l3ge2: the terms of tpL_bwd with output order
//   l3 <= 1 / l3 = 2 (their sum is tpL_bwd)
// V and G hold one channel's (l_max+1)^2 components, index l*l + (m + l).
// T is grouped by output order l3: block l3 starts at TPL_TOFF[l3] and holds
// TPL_P[l3] paths (in lexicographic path order) of 2 l3 + 1 components each.
//
// For l_max in {1, 2} also the full-O(3) product over inputs of both
// parities s (0: true tensors, (-1)^l under inversion; 1: pseudotensors):
//   tpLo_fwd(V, G, T), tpLo_bwd(V, G, dT, dV, dG)
// with V holding 2 (l_max+1)^2 components, index s (l_max+1)^2 + l*l + m + l,
// and G the (true-tensor) neighbour sums as above.  Every path (s1, l1, l2)
// -> (l3, s3), s3 = (l1 + s1 + l2 + l3) mod 2, of the even and odd couplings;
// T grouped by output block b = s3 (l_max+1) + l3 (tpLo_P(b), tpLo_toff(b)),
// paths in (s1, l1, l2) order inside a block.  Block 0 (true scalars) holds
// exactly the natural-parity scalar paths in the same order, so the scalar
// functions tpL_fwd_scalar / tpL_bwd_scalar serve the full-O(3) model too.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

namespace {

// Real spherical harmonics in component normalisation (sum_m Y^2 = 2l+1),
// m = -l..l, closed forms for l <= 2.
void sh(double x, double y, double z, double* Y) {
  const double s3 = std::sqrt(3.0), s5 = std::sqrt(5.0), s15 = std::sqrt(15.0);
  Y[0] = 1.0;
  Y[1] = s3 * y;
  Y[2] = s3 * z;
  Y[3] = s3 * x;
  Y[4] = s15 * x * y;
  Y[5] = s15 * y * z;
  Y[6] = 0.5 * s5 * (3.0 * z * z - 1.0);
  Y[7] = s15 * x * z;
  Y[8] = 0.5 * s15 * (x * x - y * y);
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  const double pi = std::acos(-1.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (t * p1 - p0) / (t * t - 1.0);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

struct Path {
  int l1, l2, l3;
  std::vector<double> c;  // (2l1+1)(2l2+1)(2l3+1)
  int s1 = 0;             // parity of the V input (full-O(3) tables)
};

// Gradients of the harmonic polynomials R_lm (l = 1, 2; the closed forms of
// sh() with 3z^2 - 1 read as 2z^2 - x^2 - y^2) at (x, y, z): g[m][axis].
void grad_r(int l, double x, double y, double z, double g[5][3]) {
  const double s3 = std::sqrt(3.0), s5 = std::sqrt(5.0), s15 = std::sqrt(15.0);
  const double g1[3][3] = {{0.0, s3, 0.0}, {0.0, 0.0, s3}, {s3, 0.0, 0.0}};
  const double g2[5][3] = {{s15 * y, s15 * x, 0.0},
                           {0.0, s15 * z, s15 * y},
                           {-s5 * x, -s5 * y, 2.0 * s5 * z},
                           {s15 * z, 0.0, s15 * x},
                           {s15 * x, -s15 * y, 0.0}};
  for (int m = 0; m < 2 * l + 1; ++m)
    for (int a = 0; a < 3; ++a) g[m][a] = l == 1 ? g1[m][a] : g2[m][a];
}

Path normalise_odd(Path p) {
  double nrm = 0.0;
  for (double v : p.c) nrm += v * v;
  nrm = std::sqrt(nrm);
  if (!(nrm > 1e-8)) {
    std::fprintf(stderr, "gen_tp: odd coupling (%d, %d, %d) vanished\n", p.l1, p.l2, p.l3);
    std::exit(1);
  }
  for (double& v : p.c) v /= nrm;
  for (double& v : p.c)
    if (std::fabs(v) < 1e-13) v = 0.0;
  for (double v : p.c)
    if (std::fabs(v) > 1e-12) {
      if (v < 0)
        for (double& w : p.c) w = -w;
      break;
    }
  return p;
}

// Coupling tensor of an odd path (l1, l2 >= 1 there: with l1 = 0 or l2 = 0
// the triangle forces l3 = l2 or l1, an even sum).
Path coupling_odd(int l1, int l2, int l3) {
  Path p{l1, l2, l3, {}};
  const int n1 = 2 * l1 + 1, n2 = 2 * l2 + 1, n3 = 2 * l3 + 1;
  if (l1 < 1 || l2 < 1 || l1 > 2 || l2 > 2) {
    std::fprintf(stderr, "gen_tp: odd path (%d, %d, %d) out of range\n", l1, l2, l3);
    std::exit(1);
  }
  p.c.assign(n1 * n2 * n3, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(8, gx, gw);
  const int nphi = 16;
  const double pi = std::acos(-1.0);
  double Y[9], ga[5][3], gb[5][3];
  for (size_t a = 0; a < gx.size(); ++a) {
    const double ct = gx[a], st = std::sqrt(1.0 - ct * ct);
    for (int b = 0; b < nphi; ++b) {
      const double ph = 2.0 * pi * b / nphi;
      const double u[3] = {st * std::cos(ph), st * std::sin(ph), ct};
      sh(u[0], u[1], u[2], Y);
      grad_r(l1, u[0], u[1], u[2], ga);
      grad_r(l2, u[0], u[1], u[2], gb);
      const double wt = gw[a] * (2.0 * pi / nphi);
      for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j) {
          const double cx = ga[i][1] * gb[j][2] - ga[i][2] * gb[j][1];
          const double cy = ga[i][2] * gb[j][0] - ga[i][0] * gb[j][2];
          const double cz = ga[i][0] * gb[j][1] - ga[i][1] * gb[j][0];
          const double tri = u[0] * cx + u[1] * cy + u[2] * cz;
          for (int k = 0; k < n3; ++k) p.c[(i * n2 + j) * n3 + k] += wt * tri * Y[l3 * l3 + k];
        }
    }
  }
  return normalise_odd(p);
}

Path coupling(int l1, int l2, int l3) {
  Path p{l1, l2, l3, {}};
  const int n1 = 2 * l1 + 1, n2 = 2 * l2 + 1, n3 = 2 * l3 + 1;
  p.c.assign(n1 * n2 * n3, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(8, gx, gw);
  const int nphi = 16;
  const double pi = std::acos(-1.0);
  double Y[9];
  for (size_t a = 0; a < gx.size(); ++a) {
    const double ct = gx[a], st = std::sqrt(1.0 - ct * ct);
    for (int b = 0; b < nphi; ++b) {
      const double ph = 2.0 * pi * b / nphi;
      sh(st * std::cos(ph), st * std::sin(ph), ct, Y);
      const double wt = gw[a] * (2.0 * pi / nphi);
      for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j)
          for (int k = 0; k < n3; ++k)
            p.c[(i * n2 + j) * n3 + k] +=
                wt * Y[l1 * l1 + i] * Y[l2 * l2 + j] * Y[l3 * l3 + k];
    }
  }
  double nrm = 0.0;
  for (double v : p.c) nrm += v * v;
  nrm = std::sqrt(nrm);
  for (double& v : p.c) v /= nrm;
  // sign: C(Y_l1(z), Y_l2(z)) . Y_l3(z) > 0
  sh(0.0, 0.0, 1.0, Y);
  double s = 0.0;
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j)
      for (int k = 0; k < n3; ++k)
        s += p.c[(i * n2 + j) * n3 + k] * Y[l1 * l1 + i] * Y[l2 * l2 + j] *
             Y[l3 * l3 + k];
  if (s < 0)
    for (double& v : p.c) v = -v;
  for (double& v : p.c)
    if (std::fabs(v) < 1e-13) v = 0.0;
  return p;
}

std::string lit(double v) {
  char buf[64];
  std::snprintf(buf, sizeof buf, "%.9ef", v);
  return buf;
}

void emit(FILE* f, int lmax, bool o3) {
  std::vector<Path> paths;
  std::vector<int> blk;   // output block of every path: s3 (l_max + 1) + l3
  for (int s1 = 0; s1 <= (o3 ? 1 : 0); ++s1)
    for (int l1 = 0; l1 <= lmax; ++l1)
      for (int l2 = 0; l2 <= lmax; ++l2)
        for (int l3 = std::abs(l1 - l2); l3 <= std::min(l1 + l2, lmax); ++l3) {
          const int odd = (l1 + l2 + l3) % 2;
          if (odd && !o3) continue;
          paths.push_back(odd ? coupling_odd(l1, l2, l3) : coupling(l1, l2, l3));
          paths.back().s1 = s1;
          blk.push_back(((l1 + s1 + l2 + l3) % 2) * (lmax + 1) + l3);
        }
  const int nblk = o3 ? 2 * (lmax + 1) : lmax + 1;
  const int nlm = (lmax + 1) * (lmax + 1);
  std::vector<int> P(nblk, 0), toff(nblk, 0);
  for (int b : blk) P[b]++;
  int nt = 0;
  for (int b = 0; b < nblk; ++b) {
    toff[b] = nt;
    nt += P[b] * (2 * (b % (lmax + 1)) + 1);
  }
  // output index of every path's first component
  std::vector<int> base(paths.size());
  {
    std::vector<int> q(nblk, 0);
    for (size_t i = 0; i < paths.size(); ++i) {
      const int b = blk[i];
      base[i] = toff[b] + q[b] * (2 * paths[i].l3 + 1);
      q[b]++;
    }
  }
  const std::string L = std::to_string(lmax) + (o3 ? "o" : "");
  const std::string U = std::to_string(lmax) + (o3 ? "O" : "");
  std::fprintf(f, "// ---- l_max = %d%s: %zu paths\n", lmax, o3 ? ", full O(3)" : "", paths.size());
  std::fprintf(f, "#define TP%s_NT %d\n#define TP%s_NS %d\n", U.c_str(), nt, U.c_str(), P[0]);
  std::fprintf(f, "__host__ __device__ constexpr int tp%s_P(int l) { return ", L.c_str());
  for (int b = 0; b < nblk; ++b) std::fprintf(f, "l == %d ? %d : ", b, P[b]);
  std::fprintf(f, "0; }\n");
  std::fprintf(f, "__host__ __device__ constexpr int tp%s_toff(int l) { return ", L.c_str());
  for (int b = 0; b < nblk; ++b) std::fprintf(f, "l == %d ? %d : ", b, toff[b]);
  std::fprintf(f, "0; }\n");
  // term lists
  struct Term { int o, a, b; double c; };
  std::vector<Term> terms, sterms;
  for (size_t i = 0; i < paths.size(); ++i) {
    const Path& p = paths[i];
    const int n2 = 2 * p.l2 + 1, n3 = 2 * p.l3 + 1;
    for (int a = 0; a < 2 * p.l1 + 1; ++a)
      for (int b = 0; b < n2; ++b)
        for (int k = 0; k < n3; ++k) {
          double c = p.c[(a * n2 + b) * n3 + k];
          if (c == 0.0) continue;
          Term t{base[i] + k, p.s1 * nlm + p.l1 * p.l1 + a, p.l2 * p.l2 + b, c};
          terms.push_back(t);
          if (blk[i] == 0) sterms.push_back(t);
        }
  }
  std::fprintf(f, "#define TP%s_NNZ %zu\n", U.c_str(), terms.size());
  auto fwd = [&](const char* name, const std::vector<Term>& ts, int nout) {
    std::fprintf(f, "template <class S>\n__device__ __forceinline__ void tp%s_%s(const S* __restrict__ V, "
                 "const S* __restrict__ G, S* __restrict__ T) {\n", L.c_str(), name);
    for (int o = 0; o < nout; ++o) {
      std::string e;
      for (auto& t : ts)
        if (t.o == o) {
          std::string term = lit(t.c) + " * V[" + std::to_string(t.a) + "] * G[" +
                             std::to_string(t.b) + "]";
          e = e.empty() ? term : e + " + " + term;
        }
      std::fprintf(f, "  T[%d] = %s;\n", o, e.empty() ? "S(0.0f)" : e.c_str());
    }
    std::fprintf(f, "}\n");
  };
  // Adjoint: with M[a][b] = sum_o c_abo dT[o] (one entry per (a, b) that has
  // terms), dV[a] += sum_b M[a][b] G[b] and dG[b] += sum_a M[a][b] V[a]: each
  // CG term costs one multiply-add in M instead of one in each of dV and dG.
  // Emitted row by row (a), so that only one row of M is live at a time.
  auto bwd = [&](const char* name, const std::vector<Term>& ts) {
    std::fprintf(f, "template <class S>\n__device__ __forceinline__ void tp%s_%s(const S* __restrict__ V, "
                 "const S* __restrict__ G, const S* __restrict__ dT, "
                 "S* __restrict__ dV, S* __restrict__ dG) {\n", L.c_str(), name);
    const int nv = o3 ? 2 * nlm : nlm;
    for (int a = 0; a < nv; ++a) {
      std::vector<int> bs;
      std::string block;
      for (int b = 0; b < nlm; ++b) {
        std::string e;
        for (auto& t : ts)
          if (t.a == a && t.b == b) {
            const std::string term = lit(t.c) + " * dT[" + std::to_string(t.o) + "]";
            e = e.empty() ? term : e + " + " + term;
          }
        if (e.empty()) continue;
        bs.push_back(b);
        block += "    const S m" + std::to_string(b) + " = " + e + ";\n";
      }
      if (bs.empty()) continue;
      std::string dv;
      for (int b : bs) {
        const std::string term = "m" + std::to_string(b) + " * G[" + std::to_string(b) + "]";
        dv = dv.empty() ? term : dv + " + " + term;
      }
      block += "    dV[" + std::to_string(a) + "] += " + dv + ";\n";
      for (int b : bs)
        block += "    dG[" + std::to_string(b) + "] += m" + std::to_string(b) + " * V[" + std::to_string(a) + "];\n";
      std::fprintf(f, "  {\n%s  }\n", block.c_str());
    }
    std::fprintf(f, "}\n");
  };
  fwd("fwd", terms, nt);
  if (o3) {         // scalars: block 0 is the natural-parity scalar block
    bwd("bwd", terms);
    return;
  }
  fwd("fwd_scalar", sterms, P[0]);
  bwd("bwd", terms);
  bwd("bwd_scalar", sterms);
  // the adjoint split by output order (l3 <= 1, l3 = 2): the two halves add
  // up to tpL_bwd and read only their own entries of dT
  std::vector<Term> lo, hi;
  for (auto& t : terms) (t.o < toff[std::min(2, lmax)] || lmax < 2 ? lo : hi).push_back(t);
  bwd("bwd_l3lt2", lo);
  bwd("bwd_l3ge2", hi);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 2) {
    std::fprintf(stderr, "usage: gen_tp OUT.inc\n");
    return 2;
  }
  FILE* f = std::fopen(argv[1], "w");
  if (!f) return 1;
  std::fprintf(f, "// Generated by gen_tp.cpp at build time; do not edit.\n#pragma once\n");
  emit(f, 0, false);
  emit(f, 1, false);
  emit(f, 2, false);
  emit(f, 1, true);
  emit(f, 2, true);
  std::fclose(f);
  return 0;
}
