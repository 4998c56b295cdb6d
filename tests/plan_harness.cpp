// Host harness for the planner of the shifted systems (plan_systems): reads
// "form fuse conj k", then k lines "c_re c_im b_re b_im" (one function), then
// "a0", and prints the base and, per system, "node quad cr ci u1r u1i u2r u2i
// wr wi gr gi ar ai br bi yr yi xr xi" for function 0.  Driven by
// test_plan.py.
#include <cstdio>
#include <cstring>

#include "../paper_2210_03714_gb300/csrc/fm_job.h"

int main() {
  int form, fuse, conj, k;
  if (std::scanf("%d %d %d %d", &form, &fuse, &conj, &k) != 4) return 1;
  fmk::FmCoef cf;
  std::memset(&cf, 0, sizeof cf);
  cf.k = k;
  cf.nfun = 1;
  cf.conj_pair = conj;
  for (int i = 0; i < k; ++i)
    if (std::scanf("%lf %lf %lf %lf", &cf.c_re[i], &cf.c_im[i], &cf.b_re[0][i], &cf.b_im[0][i]) != 4)
      return 1;
  if (std::scanf("%lf", &cf.a0[0]) != 1) return 1;
  fmk::Sys sys[fmk::kMaxTerms];
  double base[2];
  const int ns = fmk::plan_systems(cf, form, fuse != 0, sys, base);
  std::printf("%d %.17g\n", ns, base[0]);
  for (int q = 0; q < ns; ++q) {
    const fmk::Sys& S = sys[q];
    std::printf("%d %d %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g "
                "%.17g %.17g %.17g %.17g %.17g\n",
                S.node, S.quad, S.cr, S.ci, S.u1r, S.u1i, S.u2r, S.u2i, S.wr[0], S.wi[0], S.gr[0],
                S.gi[0], S.ar[0], S.ai[0], S.br[0], S.bi[0], S.yr[0], S.yi[0], S.xr[0], S.xi[0]);
  }
  return 0;
}
