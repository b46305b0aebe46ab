// Persistent autotuner results: one text line per (device, grid, precision, batch) with the apply
// launch shape the autotuner picked, so that a later process (or a profiler run, whose serialised
// cold-cache timings would pick differently) reuses the choice instead of timing the candidates
// again.  Host code only.
//
// Line format (whitespace separated; the last matching line of a file wins):
//   fit-tune 1 <device> <sm_count> <nx> <ny> <nz> <prec> <nbatch> <variant_count> <choice>
// <device> is the CUDA device name with blanks replaced by '_'; <variant_count> is the number of
// fused variants this build compiles for <prec>, so that a file written by a build with another
// variant table is ignored; <choice> is -1 (generic kernel) or a fused variant index.
#include <cstdio>
#include <cstring>
#include <string>

#include "fit_internal.cuh"

namespace {

std::string sanitize(const char* s) {
  std::string o(s ? s : "");
  for (char& c : o)
    if (c == ' ' || c == '\t' || c == '\n' || c == '\r') c = '_';
  return o.empty() ? std::string("_") : o;
}

}  // namespace

extern "C" {

fit_status fit_tuning_record(const char* path, const char* device, int sm_count, int nx, int ny, int nz, fit_prec prec,
                             int nbatch, int choice) {
  FIT_REQUIRE(path && *path && device, "fit_tuning_record: null argument");
  FIT_REQUIRE(prec == FIT_C64 || prec == FIT_C128, "fit_tuning_record: unknown precision");
  FIT_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1 && nbatch >= 1 && sm_count >= 1, "fit_tuning_record: bad key");
  const int nvar = fit_apply_variant_count(prec);
  FIT_REQUIRE(choice >= -1 && choice < nvar, "fit_tuning_record: choice out of range");
  FILE* f = std::fopen(path, "a");
  if (!f) {
    fit_set_error(std::string("fit_tuning_record: cannot open ") + path);
    return FIT_EINVAL;
  }
  const int n = std::fprintf(f, "fit-tune 1 %s %d %d %d %d %d %d %d %d\n", sanitize(device).c_str(), sm_count, nx, ny,
                             nz, (int)prec, nbatch, nvar, choice);
  const int closed = std::fclose(f);
  if (n < 0 || closed != 0) {
    fit_set_error(std::string("fit_tuning_record: write failed on ") + path);
    return FIT_EINVAL;
  }
  return FIT_OK;
}

fit_status fit_tuning_lookup(const char* path, const char* device, int sm_count, int nx, int ny, int nz, fit_prec prec,
                             int nbatch, int* choice) {
  FIT_REQUIRE(path && device && choice, "fit_tuning_lookup: null argument");
  FIT_REQUIRE(prec == FIT_C64 || prec == FIT_C128, "fit_tuning_lookup: unknown precision");
  *choice = -2;
  FILE* f = std::fopen(path, "r");
  if (!f) return FIT_OK;  // no cache yet
  const std::string dev = sanitize(device);
  const int nvar = fit_apply_variant_count(prec);
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    char tag[16], name[256];
    int ver, sms, lx, ly, lz, lp, lb, lv, lc;
    if (std::sscanf(line, "%15s %d %255s %d %d %d %d %d %d %d %d", tag, &ver, name, &sms, &lx, &ly, &lz, &lp, &lb, &lv,
                    &lc) != 11)
      continue;  // malformed or foreign line
    if (std::strcmp(tag, "fit-tune") != 0 || ver != 1) continue;
    if (dev != name || sms != sm_count || lx != nx || ly != ny || lz != nz || lp != (int)prec || lb != nbatch) continue;
    if (lv != nvar || lc < -1 || lc >= nvar) continue;  // another build's variant table, or out of range
    *choice = lc;
  }
  std::fclose(f);
  return FIT_OK;
}

}  // extern "C"

// The device key of the current device: name with blanks replaced, and its SM count.
fit_status fit_tuning_device_key(std::string* name, int* sm_count) {
  int dev = 0;
  FIT_CHECK_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  FIT_CHECK_CUDA(cudaGetDeviceProperties(&prop, dev));
  *name = sanitize(prop.name);
  *sm_count = prop.multiProcessorCount;
  return FIT_OK;
}
