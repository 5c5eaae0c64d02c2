// Autotuner table of the split-precision products (see tune.h): an in-memory map per GPU
// model, loaded once from the cache file and appended to as new shapes are measured.  Each
// line: gpu-name|M N K krule lower transA transB inplace precision choice ms_f32 ms_wide ms_square
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <sys/stat.h>
#include <tuple>
#include "tune.h"

namespace glasso {

bool GemmShape::operator<(const GemmShape& o) const {
  return std::tie(M, N, K, krule, lower, transA, transB, inplace, precision) <
         std::tie(o.M, o.N, o.K, o.krule, o.lower, o.transA, o.transB, o.inplace, o.precision);
}

GemmShape GemmShape::of(const GemmArgs& a, int precision) {
  GemmShape s;
  s.M = a.M;
  s.N = a.N;
  s.K = a.K;
  s.krule = a.krule;
  s.lower = a.lower;
  s.transA = a.transA;
  s.transB = a.transB;
  s.inplace = (a.C == a.A || a.C == a.B) ? 1 : 0;
  s.precision = precision;
  return s;
}

namespace {
std::mutex g_mu;
bool g_loaded = false;
std::map<std::pair<std::string, GemmShape>, GemmChoice> g_table;

std::string cache_path() {
  const char* p = std::getenv("GLASSO_TUNE_CACHE");
  if (p) return std::string(p) == "off" ? std::string() : std::string(p);
  const char* home = std::getenv("HOME");
  return home ? std::string(home) + "/.cache/glasso_gemm_tune.txt" : std::string();
}

void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const std::string path = cache_path();
  if (path.empty()) return;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t bar = line.find('|');
    if (bar == std::string::npos) continue;
    std::istringstream in(line.substr(bar + 1));
    GemmShape s;
    int c = 0;
    if (!(in >> s.M >> s.N >> s.K >> s.krule >> s.lower >> s.transA >> s.transB >> s.inplace >> s.precision >> c))
      continue;
    if (c < 0 || c > 3) continue;
    g_table[{line.substr(0, bar), s}] = (GemmChoice)c;
  }
}
}  // namespace

GemmChoice tuned_choice(const std::string& gpu, const GemmShape& s) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  auto it = g_table.find({gpu, s});
  return it == g_table.end() ? GemmChoice::Default : it->second;
}

bool tuned(const std::string& gpu, const GemmShape& s) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  return g_table.count({gpu, s}) != 0;
}

void record_choice(const std::string& gpu, const GemmShape& s, GemmChoice c, const double ms[4]) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  g_table[{gpu, s}] = c;
  const std::string path = cache_path();
  if (path.empty()) return;
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    const std::string dir = path.substr(0, slash);
    std::string cmd;  // create the directory without a shell: mkdir each prefix
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') {
        cmd = dir.substr(0, i);
        if (!cmd.empty()) (void)::mkdir(cmd.c_str(), 0755);
      }
  }
  std::ofstream f(path, std::ios::app);
  if (!f) return;
  f << gpu << '|' << s.M << ' ' << s.N << ' ' << s.K << ' ' << s.krule << ' ' << s.lower << ' ' << s.transA << ' '
    << s.transB << ' ' << s.inplace << ' ' << s.precision << ' ' << (int)c << ' ' << ms[1] << ' ' << ms[2] << ' '
    << ms[3] << '\n';
}

}  // namespace glasso
