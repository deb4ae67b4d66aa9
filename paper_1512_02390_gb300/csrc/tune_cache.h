// Cache of the launch-shape autotuner: one JSON object per line,
//   {"key": "<device>|p=16|n_o=2|prec=2|var=0|elems=64x64", "fuse": 0, "spw": 1, "tc": 1, "eo": 0, "us": 123.4}
// keyed by the device name and what the timed kernels depend on (level order,
// overlap, precision, operator kind, element grid of the level).
#pragma once

#include <string>

namespace sem {

struct TuneVal {
  int fuse = 0;     // scatter fused into the level residual
  int spw = 1;      // mma.sync sweep: subdomains per warp
  int tc = 0;       // 1: reduced-precision sweep on tcgen05 (stacked subdomains)
  int eo = -1;      // level residual: -1 even-odd in FP64 only, 0 plain, 1 even-odd
  double us = 0.0;  // measured time of the chosen down-sweep step
};

std::string tune_key(const std::string& device, int p, int n_o, int precision, int var, int ex, int ey);
// false if the file or the key is absent (or the line does not parse)
bool tune_cache_find(const std::string& path, const std::string& key, TuneVal& v);
// insert or replace the key; returns "" or an error message
std::string tune_cache_store(const std::string& path, const std::string& key, const TuneVal& v);

}  // namespace sem
