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
#include <cmath>
#include <cstdio>
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
};

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

void emit(FILE* f, int lmax) {
  std::vector<Path> paths;
  for (int l1 = 0; l1 <= lmax; ++l1)
    for (int l2 = 0; l2 <= lmax; ++l2)
      for (int l3 = std::abs(l1 - l2); l3 <= std::min(l1 + l2, lmax); ++l3)
        if ((l1 + l2 + l3) % 2 == 0) paths.push_back(coupling(l1, l2, l3));
  int P[3] = {0, 0, 0}, toff[3] = {0, 0, 0};
  for (auto& p : paths) P[p.l3]++;
  int nt = 0;
  for (int l = 0; l <= lmax; ++l) {
    toff[l] = nt;
    nt += P[l] * (2 * l + 1);
  }
  // output index of every path's first component
  std::vector<int> base(paths.size());
  {
    int q[3] = {0, 0, 0};
    for (size_t i = 0; i < paths.size(); ++i) {
      int l3 = paths[i].l3;
      base[i] = toff[l3] + q[l3] * (2 * l3 + 1);
      q[l3]++;
    }
  }
  const std::string L = std::to_string(lmax);
  std::fprintf(f, "// ---- l_max = %d: %zu paths\n", lmax, paths.size());
  std::fprintf(f, "#define TP%d_NT %d\n#define TP%d_NS %d\n", lmax, nt, lmax, P[0]);
  std::fprintf(f, "__host__ __device__ constexpr int tp%d_P(int l) { return ", lmax);
  for (int l = 0; l <= lmax; ++l) std::fprintf(f, "l == %d ? %d : ", l, P[l]);
  std::fprintf(f, "0; }\n");
  std::fprintf(f, "__host__ __device__ constexpr int tp%d_toff(int l) { return ", lmax);
  for (int l = 0; l <= lmax; ++l) std::fprintf(f, "l == %d ? %d : ", l, toff[l]);
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
          Term t{base[i] + k, p.l1 * p.l1 + a, p.l2 * p.l2 + b, c};
          terms.push_back(t);
          if (p.l3 == 0) sterms.push_back(t);
        }
  }
  std::fprintf(f, "#define TP%d_NNZ %zu\n", lmax, terms.size());
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
    const int nc = (lmax + 1) * (lmax + 1);
    for (int a = 0; a < nc; ++a) {
      std::vector<int> bs;
      std::string block;
      for (int b = 0; b < nc; ++b) {
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
  emit(f, 0);
  emit(f, 1);
  emit(f, 2);
  std::fclose(f);
  return 0;
}
