// JSON-lines cache of the launch-shape autotuner (tune_cache.h).
#include "tune_cache.h"

#include <cstdio>
#include <fstream>
#include <sstream>
#include <vector>

namespace sem {

namespace {

// the fields of one cache line; false if it does not have the written form
bool parse_line(const std::string& line, std::string& key, TuneVal& v) {
  const std::string k0 = "{\"key\": \"";
  if (line.compare(0, k0.size(), k0) != 0) return false;
  const size_t e = line.find('"', k0.size());
  if (e == std::string::npos) return false;
  key = line.substr(k0.size(), e - k0.size());
  TuneVal t;
  if (std::sscanf(line.c_str() + e, "\", \"fuse\": %d, \"spw\": %d, \"tc\": %d, \"eo\": %d, \"us\": %lf}", &t.fuse,
                  &t.spw, &t.tc, &t.eo, &t.us) != 5)
    return false;
  if (t.fuse < 0 || t.fuse > 1 || t.spw < 1 || t.spw > 64 || t.tc < 0 || t.tc > 1 || t.eo < -1 || t.eo > 1)
    return false;
  v = t;
  return true;
}

std::string format_line(const std::string& key, const TuneVal& v) {
  char buf[128];
  std::snprintf(buf, sizeof(buf), "\", \"fuse\": %d, \"spw\": %d, \"tc\": %d, \"eo\": %d, \"us\": %.3f}", v.fuse,
                v.spw, v.tc, v.eo, v.us);
  return "{\"key\": \"" + key + buf;
}

}  // namespace

std::string tune_key(const std::string& device, int p, int n_o, int precision, int var, int ex, int ey) {
  std::ostringstream o;
  std::string dev;
  for (char c : device) dev += (c == '"' || c == '\\' || c == '|') ? '_' : c;
  o << dev << "|p=" << p << "|n_o=" << n_o << "|prec=" << precision << "|var=" << var << "|elems=" << ex << "x"
    << ey;
  return o.str();
}

bool tune_cache_find(const std::string& path, const std::string& key, TuneVal& v) {
  std::ifstream in(path);
  if (!in) return false;
  std::string line, k;
  TuneVal t;
  bool found = false;
  while (std::getline(in, line))
    if (parse_line(line, k, t) && k == key) {
      v = t;  // the last entry of a key wins
      found = true;
    }
  return found;
}

std::string tune_cache_store(const std::string& path, const std::string& key, const TuneVal& v) {
  std::vector<std::string> keep;
  {
    std::ifstream in(path);
    std::string line, k;
    TuneVal t;
    while (in && std::getline(in, line))
      if (parse_line(line, k, t) && k != key) keep.push_back(line);
  }
  keep.push_back(format_line(key, v));
  const std::string tmp = path + ".tmp";
  {
    std::ofstream out(tmp, std::ios::trunc);
    if (!out) return "cannot write " + tmp;
    for (const auto& l : keep) out << l << "\n";
    if (!out) return "cannot write " + tmp;
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) return "cannot rename " + tmp + " to " + path;
  return "";
}

}  // namespace sem
