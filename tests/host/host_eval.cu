// Host-side evaluator for one generated process unit: reads the parameter block and FP64 momenta,
// writes the FP64 and the mixed-precision |M|^2 of every point.  Built by tests/test_host_programs.py
// with -DGEN_UNIT="<unit without its kernel registration>" -DTAG=<process symbol> -DNEXT_H=<legs>.
//
// input : int32 n, int32 n_params, double params[n_params], double momenta[n][NEXT_H][4]
// output: double out[n][2] = (FP64 path, mixed path)
#include <cstdio>
#include <cstring>
#include <vector>
#include GEN_UNIT

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  int n = 0, npar = 0;
  if (fread(&n, 4, 1, f) != 1 || fread(&npar, 4, 1, f) != 1 || n < 0 || npar < 0) return 1;
  std::vector<double> par(npar), mom((size_t)n * NEXT_H * 4);
  if ((int)fread(par.data(), 8, npar, f) != npar) return 1;
  if (fread(mom.data(), 8, mom.size(), f) != mom.size()) return 1;
  fclose(f);
  me::TAG::Traits::Params prm;
  if (sizeof(prm) != par.size() * sizeof(double)) return 2;  // the block is all doubles, in order
  std::memcpy(&prm, par.data(), sizeof(prm));
  const auto mx = me::TAG::Traits::mixed_params(prm);
  std::vector<double> out((size_t)n * 2);
  for (int i = 0; i < n; ++i) {
    double pd[NEXT_H][4];
    me::df pm[NEXT_H][4];
    for (int k = 0; k < NEXT_H; ++k)
      for (int m = 0; m < 4; ++m) {
        pd[k][m] = mom[((size_t)i * NEXT_H + k) * 4 + m];
        pm[k][m] = me::from_double(pd[k][m]);
      }
    out[2 * (size_t)i] = me::TAG::Traits::eval64(pd, prm);
    out[2 * (size_t)i + 1] = me::TAG::Traits::evalmx(pm, mx);
  }
  f = fopen(argv[2], "wb");
  if (!f) return 1;
  const bool ok = fwrite(out.data(), 8, out.size(), f) == out.size();
  fclose(f);
  return ok ? 0 : 1;
}
