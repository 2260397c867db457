// Launch-shape autotuner (see lma_tune.cuh).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "lma_impl.cuh"
#include "lma_tune.cuh"

namespace lma {
namespace tune {

namespace {

struct Entry {
  int choice = 0;
  std::vector<std::pair<int, float>> ms;  // candidate, milliseconds per launch (empty: read from the file)
};

struct State {
  std::mutex mu;
  int enabled = -1;                                    // -1: not read from the environment yet
  std::map<int, std::map<std::string, Entry>> cache;  // device -> key -> entry
  std::map<int, std::string> dev_name;
  std::vector<std::pair<std::string, int>> pins;      // key prefix -> forced choice
  bool file_read = false;
};

State& st() {
  static State s;
  return s;
}

std::string device_name(State& s, int dev) {
  auto it = s.dev_name.find(dev);
  if (it != s.dev_name.end()) return it->second;
  cudaDeviceProp p;
  std::string name = "device";
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) name = p.name;
  for (char& c : name)
    if (c == '|' || c == '\n') c = ' ';
  s.dev_name[dev] = name;
  return name;
}

const char* cache_file() {
  const char* f = getenv("LMA_TUNE_CACHE");
  return (f && f[0]) ? f : nullptr;
}

// Lines "device name|key|choice" of the cache file, for every device whose name matches.
void read_file(State& s) {
  if (s.file_read) return;
  s.file_read = true;
  const char* path = cache_file();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) ndev = 0;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    std::string l(line);
    while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
    const size_t a = l.find('|'), b = l.rfind('|');
    if (a == std::string::npos || b == a) continue;
    const std::string dn = l.substr(0, a), key = l.substr(a + 1, b - a - 1);
    const int choice = atoi(l.c_str() + b + 1);
    for (int d = 0; d < ndev; ++d)
      if (device_name(s, d) == dn) s.cache[d][key].choice = choice;
  }
  fclose(f);
}

void append_file(const std::string& dn, const std::string& key, int choice) {
  const char* path = cache_file();
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s|%s|%d\n", dn.c_str(), key.c_str(), choice);
  fclose(f);
}

}  // namespace

bool enabled() {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  if (s.enabled < 0) {
    const char* e = getenv("LMA_AUTOTUNE");
    s.enabled = (e && e[0] == '0') ? 0 : 1;
  }
  return s.enabled == 1;
}

void set_enabled(bool on) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  s.enabled = on ? 1 : 0;
}

int pick(const std::string& key, const std::vector<int>& cands, int fallback, cudaStream_t stream,
         const std::function<void(int)>& run, int reps) {
  if (cands.empty()) return fallback;
  if (cands.size() == 1) return cands[0];
  State& s = st();
  {
    std::lock_guard<std::mutex> lk(s.mu);
    for (auto it = s.pins.rbegin(); it != s.pins.rend(); ++it)
      if (key.compare(0, it->first.size(), it->first) == 0)
        for (int c : cands)
          if (c == it->second) return c;
  }
  if (!enabled()) return fallback;
  int dev = 0;
  LMA_CK(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(s.mu);
    read_file(s);
    auto& m = s.cache[dev];
    auto it = m.find(key);
    if (it != m.end()) return it->second.choice;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  LMA_CK(cudaEventCreate(&a));
  LMA_CK(cudaEventCreate(&b));
  Entry e;
  float best = 0.f;
  try {
    for (int c : cands) {
      run(c);  // warm-up (also loads the kernel)
      LMA_CK(cudaEventRecord(a, stream));
      for (int r = 0; r < reps; ++r) run(c);
      LMA_CK(cudaEventRecord(b, stream));
      LMA_CK(cudaEventSynchronize(b));
      float ms = 0.f;
      LMA_CK(cudaEventElapsedTime(&ms, a, b));
      ms /= (float)reps;
      e.ms.emplace_back(c, ms);
      if (e.ms.size() == 1 || ms < best) {
        best = ms;
        e.choice = c;
      }
    }
  } catch (...) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    throw;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::lock_guard<std::mutex> lk(s.mu);
  s.cache[dev][key] = e;
  append_file(device_name(s, dev), key, e.choice);
  return e.choice;
}

std::string report() {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  std::ostringstream o;
  for (auto& dv : s.cache)
    for (auto& kv : dv.second) {
      o << device_name(s, dv.first) << " | " << kv.first << " | " << kv.second.choice << " |";
      for (auto& cm : kv.second.ms) o << " " << cm.first << ":" << cm.second;
      o << "\n";
    }
  return o.str();
}

void pin(const char* prefix, int choice) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  if (!prefix) {
    s.pins.clear();
    return;
  }
  s.pins.emplace_back(prefix, choice);
}

void clear() {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  s.cache.clear();
}

}  // namespace tune
}  // namespace lma
