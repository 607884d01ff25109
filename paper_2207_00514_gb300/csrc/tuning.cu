// tuning.cu -- the tuning file: for a GPU model, a dimension, a form (one
// problem or a batch) and a range of sizes, the traversal parameters the
// tuner (paper_2207_00514_gb300/tune.py) measured fastest.  Read once per
// process; the parameters only choose among exact variants of the search.
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace emst {
namespace {

struct TuneEntry {
  std::string gpu;  // device name, spaces as '_'
  int dim = 0;
  bool batched = false;
  int64_t nmin = 0, nmax = 0;
  TuneChoice c;
};

std::once_flag g_once;
std::vector<TuneEntry> g_entries;
std::mutex g_name_mu;
std::string g_names[64];

std::string tuning_path() {
  const char *e = std::getenv("EMST_TUNING_FILE");
  if (e && *e) return e;
  Dl_info info;
  if (dladdr(reinterpret_cast<void *>(&tuning_path), &info) && info.dli_fname) {
    std::string p = info.dli_fname;
    const size_t k = p.rfind('/');
    return (k == std::string::npos ? std::string(".") : p.substr(0, k)) + "/emst_tuning.txt";
  }
  return "emst_tuning.txt";
}

void load_file() {
  FILE *f = std::fopen(tuning_path().c_str(), "r");
  if (!f) return;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    if (char *h = std::strchr(line, '#')) *h = 0;
    TuneEntry t;
    int fields = 0;
    for (char *tok = std::strtok(line, " \t\r\n"); tok; tok = std::strtok(nullptr, " \t\r\n")) {
      char *eq = std::strchr(tok, '=');
      if (!eq) continue;
      *eq = 0;
      const char *k = tok, *v = eq + 1;
      if (!std::strcmp(k, "gpu")) { t.gpu = v; ++fields; }
      else if (!std::strcmp(k, "dim")) { t.dim = std::atoi(v); ++fields; }
      else if (!std::strcmp(k, "form")) { t.batched = !std::strcmp(v, "batched"); ++fields; }
      else if (!std::strcmp(k, "nmin")) { t.nmin = std::atoll(v); ++fields; }
      else if (!std::strcmp(k, "nmax")) { t.nmax = std::atoll(v); ++fields; }
      else if (!std::strcmp(k, "traversal")) t.c.traversal = std::atoi(v);
      else if (!std::strcmp(k, "block")) t.c.block = std::atoi(v);
      else if (!std::strcmp(k, "leaf")) t.c.leaf = std::atoi(v);
      else if (!std::strcmp(k, "refill")) t.c.refill = std::atoi(v);
      else if (!std::strcmp(k, "chunk")) t.c.chunk = std::atoi(v);
    }
    if (fields == 5 && t.nmax > t.nmin) g_entries.push_back(t);
  }
  std::fclose(f);
}

std::string device_name(int dev) {
  std::lock_guard<std::mutex> lock(g_name_mu);
  if (dev < 0 || dev >= 64) return std::string();
  if (g_names[dev].empty()) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
      cudaGetLastError();
      return std::string();
    }
    std::string s = prop.name;
    for (char &ch : s)
      if (ch == ' ') ch = '_';
    g_names[dev] = s;
  }
  return g_names[dev];
}

}  // namespace

bool lookup_tuning(int dim, bool batched, int64_t n, TuneChoice *out) {
  std::call_once(g_once, load_file);
  if (g_entries.empty()) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const std::string name = device_name(dev);
  for (const TuneEntry &t : g_entries) {
    if (t.gpu == name && t.dim == dim && t.batched == batched && n >= t.nmin && n < t.nmax) {
      *out = t.c;
      return true;
    }
  }
  return false;
}

}  // namespace emst
