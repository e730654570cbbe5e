// Persisted choices of the autotuners (build-side; the paper has no
// counterpart). A flat JSON object {"key": integer, ...} in the file named by
// the environment variable DSRG_AUTOTUNE_CACHE (no variable: no cache). Keys
// name what was tuned, the GPU, the precision and the size class of the
// problem; a tuner that finds its key applies the stored choice without timing
// anything, and one that times candidates stores the winner. The file is
// rewritten whole through a temporary file and a rename, so a reader never sees
// a half-written file; concurrent writers keep the last complete write.
#include <cuda_runtime.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include "internal.cuh"

namespace dsrg {
namespace {

// Parse {"k": v, ...}; returns false on anything else (the caller treats a
// malformed file as absent and overwrites it on the next store).
bool parse(const std::string& text, std::map<std::string, long long>* out) {
  size_t i = 0;
  auto ws = [&]() {
    while (i < text.size() && (text[i] == ' ' || text[i] == '\n' || text[i] == '\t' || text[i] == '\r'))
      ++i;
  };
  ws();
  if (i >= text.size() || text[i] != '{') return false;
  ++i;
  ws();
  if (i < text.size() && text[i] == '}') return true;
  while (i < text.size()) {
    ws();
    if (i >= text.size() || text[i] != '"') return false;
    const size_t k0 = ++i;
    while (i < text.size() && text[i] != '"') {
      if (text[i] == '\\') return false;
      ++i;
    }
    if (i >= text.size()) return false;
    const std::string key = text.substr(k0, i - k0);
    ++i;
    ws();
    if (i >= text.size() || text[i] != ':') return false;
    ++i;
    ws();
    const size_t v0 = i;
    if (i < text.size() && text[i] == '-') ++i;
    while (i < text.size() && text[i] >= '0' && text[i] <= '9') ++i;
    if (i == v0 || (i == v0 + 1 && text[v0] == '-')) return false;
    (*out)[key] = std::strtoll(text.c_str() + v0, nullptr, 10);
    ws();
    if (i < text.size() && text[i] == ',') {
      ++i;
      continue;
    }
    if (i < text.size() && text[i] == '}') return true;
    return false;
  }
  return false;
}

bool read_file(const char* path, std::string* text) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  char buf[4096];
  size_t n;
  text->clear();
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text->append(buf, n);
  std::fclose(f);
  return true;
}

bool valid_key(const char* key) {
  if (!key || !*key) return false;
  for (const char* c = key; *c; ++c)
    if (*c == '"' || *c == '\\' || (unsigned char)*c < 0x20) return false;
  return true;
}

}  // namespace

int tune_cache_get(const char* path, const char* key, long long* value) {
  if (!path || !valid_key(key)) return 0;
  std::string text;
  if (!read_file(path, &text)) return 0;
  std::map<std::string, long long> m;
  if (!parse(text, &m)) return -1;
  auto it = m.find(key);
  if (it == m.end()) return 0;
  *value = it->second;
  return 1;
}

bool tune_cache_put(const char* path, const char* key, long long value) {
  if (!path || !valid_key(key)) return false;
  std::map<std::string, long long> m;
  std::string text;
  if (read_file(path, &text) && !parse(text, &m)) m.clear();
  m[key] = value;
  std::string out = "{\n";
  size_t k = 0;
  for (const auto& kv : m) {
    out += "  \"" + kv.first + "\": " + std::to_string(kv.second);
    out += (++k < m.size()) ? ",\n" : "\n";
  }
  out += "}\n";
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
  if (std::fclose(f) != 0 || !ok) {
    std::remove(tmp.c_str());
    return false;
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

const char* tune_cache_path() {
  const char* p = std::getenv("DSRG_AUTOTUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

std::string tune_gpu_name(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown-gpu";
  std::string n = prop.name;
  for (char& c : n)
    if (c == '"' || c == '\\' || (unsigned char)c < 0x20) c = '_';
  return n + " sm_" + std::to_string(prop.major) + std::to_string(prop.minor);
}

// Size class of a single molecule's CCVV schedule: core orbitals rounded up to a
// multiple of 4, virtual tiles of 128, tensor-core K stages rounded up to 8,
// and the shard world (the items a rank owns).
std::string tune_size_class(const Sizes& z, int kblocks, int world) {
  const int nT = (z.nV + 127) / 128;
  return "c" + std::to_string((z.nC + 3) / 4 * 4) + "-t" + std::to_string(nT) + "-k" +
         std::to_string((kblocks + 7) / 8 * 8) + "-w" + std::to_string(world);
}

}  // namespace dsrg

extern "C" {

int32_t dsrg_tune_cache_get(const char* path, const char* key, int64_t* value) {
  if (!value) return -1;
  long long v = 0;
  const int r = dsrg::tune_cache_get(path, key, &v);
  if (r == 1) *value = (int64_t)v;
  return r;
}

dsrg_status_t dsrg_tune_cache_put(const char* path, const char* key, int64_t value) {
  if (!path || !key) return DSRG_ERR_INVALID_ARG;
  return dsrg::tune_cache_put(path, key, (long long)value) ? DSRG_OK : DSRG_ERR_INVALID_ARG;
}

}  // extern "C"
