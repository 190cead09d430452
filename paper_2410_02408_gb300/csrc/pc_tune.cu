// Launch-shape table of the single-system CG graph engine (filled by pc_autotune or
// pc_tune_set, read when a handle first builds its loop graph) and the cache file that
// persists it together with the batched launch shapes of pc_batch_autotune.
//
// Key: (block size, precision, ceil(log2 n), round(log2(nnz / n)), SM count of the current
// device).  File: one flat JSON object per line, for example
//   {"kind": "cg", "bs": 16, "prec": 1, "log2n": 21, "log2deg": 3, "sms": 152,
//    "spmv_ctas_per_sm": 4, "ring_stages": 4, "bin_pipe": -1, "fuse_update": 0, "us_per_iteration": 99.6}
//   {"kind": "batch", "n_sys": 512, "n_rows": 17886587, "nnz": 223800205, "prec": 1, "sms": 152,
//    "ctas_per_sm": 2, "team_max": 8, "setup_kb": 70, "split": 4}
// Lines that do not parse are skipped.  Host code only.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pc.h"
#include "pc_tune.h"

namespace pc {

namespace {

struct CgEntry {
  TuneKey key;
  pc_shape shape;
};

std::mutex g_tmu;
std::vector<CgEntry> g_cg;
bool g_autoloaded = false;

bool same_key(const TuneKey& a, const TuneKey& b) {
  return a.bs == b.bs && a.prec == b.prec && a.log2n == b.log2n && a.log2deg == b.log2deg && a.sms == b.sms;
}

// "key": value pairs of one flat JSON object; false when the line is not one.
bool parse_line(const std::string& line, std::map<std::string, std::string>& kv) {
  size_t i = line.find('{'), j = line.rfind('}');
  if (i == std::string::npos || j == std::string::npos || j <= i) return false;
  const std::string body = line.substr(i + 1, j - i - 1);
  size_t pos = 0;
  while (pos < body.size()) {
    const size_t q0 = body.find('"', pos);
    if (q0 == std::string::npos) break;
    const size_t q1 = body.find('"', q0 + 1);
    if (q1 == std::string::npos) return false;
    const std::string key = body.substr(q0 + 1, q1 - q0 - 1);
    const size_t colon = body.find(':', q1 + 1);
    if (colon == std::string::npos) return false;
    size_t v0 = body.find_first_not_of(" \t", colon + 1);
    if (v0 == std::string::npos) return false;
    std::string val;
    if (body[v0] == '"') {
      const size_t v1 = body.find('"', v0 + 1);
      if (v1 == std::string::npos) return false;
      val = body.substr(v0 + 1, v1 - v0 - 1);
      pos = v1 + 1;
    } else {
      size_t v1 = body.find(',', v0);
      if (v1 == std::string::npos) v1 = body.size();
      val = body.substr(v0, v1 - v0);
      while (!val.empty() && (val.back() == ' ' || val.back() == '\t')) val.pop_back();
      pos = v1;
    }
    kv[key] = val;
    const size_t comma = body.find(',', pos);
    if (comma == std::string::npos) break;
    pos = comma + 1;
  }
  return !kv.empty();
}

bool get_num(const std::map<std::string, std::string>& kv, const char* k, double* out) {
  auto it = kv.find(k);
  if (it == kv.end() || it->second.empty()) return false;
  char* end = nullptr;
  const double v = strtod(it->second.c_str(), &end);
  if (end == it->second.c_str() || *end != '\0' || !isfinite(v)) return false;
  *out = v;
  return true;
}

bool get_int(const std::map<std::string, std::string>& kv, const char* k, int64_t* out) {
  double v;
  if (!get_num(kv, k, &v) || v != floor(v) || fabs(v) > 9.0e15) return false;
  *out = (int64_t)v;
  return true;
}

void put_cg_locked(const TuneKey& k, const pc_shape& s) {
  for (CgEntry& e : g_cg)
    if (same_key(e.key, k)) {
      e.shape = s;
      return;
    }
  g_cg.push_back({k, s});
}

bool parse_cg(const std::map<std::string, std::string>& kv) {
  int64_t bs, prec, l2n, l2d, sms, ctas, ring, pipe;
  double us = 0.0;
  if (!get_int(kv, "bs", &bs) || !get_int(kv, "prec", &prec) || !get_int(kv, "log2n", &l2n) ||
      !get_int(kv, "log2deg", &l2d) || !get_int(kv, "sms", &sms) || !get_int(kv, "spmv_ctas_per_sm", &ctas) ||
      !get_int(kv, "ring_stages", &ring) || !get_int(kv, "bin_pipe", &pipe))
    return false;
  get_num(kv, "us_per_iteration", &us);
  int64_t fuse = 0;   // absent in files written before the field existed: the default
  if (kv.count("fuse_update") && !get_int(kv, "fuse_update", &fuse)) return false;
  if (bs < 1 || bs > 64 || prec < 0 || prec > 2 || ctas < 0 || ctas > 8 || ring < 0 || ring > 4 || ring == 1 ||
      pipe < -1 || pipe > 2 || fuse < 0 || fuse > 2)
    return false;
  TuneKey k{(int32_t)bs, (int32_t)prec, (int32_t)l2n, (int32_t)l2d, (int32_t)sms};
  pc_shape s;
  memset(&s, 0, sizeof(s));
  s.spmv_ctas_per_sm = (int32_t)ctas;
  s.ring_stages = (int32_t)ring;
  s.bin_pipe = (int32_t)pipe;
  s.fuse_update = (int32_t)fuse;
  s.us_per_iteration = us;
  put_cg_locked(k, s);
  return true;
}

pc_status load_locked(const char* path, int* loaded) {
  FILE* f = fopen(path, "r");
  if (!f) return PC_ERR_INVALID_ARG;
  char buf[1024];
  int n = 0;
  while (fgets(buf, sizeof buf, f)) {
    std::map<std::string, std::string> kv;
    if (!parse_line(buf, kv)) continue;
    auto kind = kv.find("kind");
    if (kind == kv.end()) continue;
    if (kind->second == "cg" && parse_cg(kv)) ++n;
    else if (kind->second == "batch" && batch_tune_parse(kv)) ++n;
  }
  fclose(f);
  if (loaded) *loaded = n;
  return PC_OK;
}

}  // namespace

int32_t current_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

TuneKey tune_key(int32_t bs, int32_t prec, int64_t n, int64_t nnz) {
  TuneKey k;
  k.bs = bs;
  k.prec = prec;
  int l = 0;
  while (l < 62 && ((int64_t)1 << l) < n) ++l;   // ceil(log2 n)
  k.log2n = l;
  const double deg = n > 0 ? (double)nnz / (double)n : 0.0;
  k.log2deg = deg > 0.0 ? (int32_t)floor(log2(deg) + 0.5) : 0;
  k.sms = current_sms();
  return k;
}

void tune_autoload() {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (g_autoloaded) return;
  g_autoloaded = true;
  const char* p = getenv("PC_TUNE_CACHE");
  if (p && p[0]) load_locked(p, nullptr);
}

bool tune_lookup(const TuneKey& k, pc_shape* out) {
  tune_autoload();
  std::lock_guard<std::mutex> lk(g_tmu);
  for (const CgEntry& e : g_cg)
    if (same_key(e.key, k)) {
      *out = e.shape;
      return true;
    }
  return false;
}

void tune_record(const TuneKey& k, const pc_shape& s) {
  std::lock_guard<std::mutex> lk(g_tmu);
  put_cg_locked(k, s);
}

pc_status tune_save_env() {
  const char* p = getenv("PC_TUNE_CACHE");
  if (!p || !p[0]) return PC_OK;
  return pc_tune_save(p);
}

}  // namespace pc

extern "C" {

pc_status pc_tune_set(int32_t block_size, int32_t prec, int64_t n, int64_t nnz, const pc_shape* shape) {
  if (!shape || block_size < 1 || block_size > 64 || prec < 0 || prec > 2 || n < 1 || nnz < 0) return PC_ERR_INVALID_ARG;
  if (shape->spmv_ctas_per_sm < 0 || shape->spmv_ctas_per_sm > 8 || shape->ring_stages < 0 || shape->ring_stages > 4 ||
      shape->ring_stages == 1 || shape->bin_pipe < -1 || shape->bin_pipe > 2 || shape->fuse_update < 0 ||
      shape->fuse_update > 2)
    return PC_ERR_INVALID_ARG;
  pc::tune_record(pc::tune_key(block_size, prec, n, nnz), *shape);
  return PC_OK;
}

int32_t pc_tune_get(int32_t block_size, int32_t prec, int64_t n, int64_t nnz, pc_shape* shape) {
  if (!shape) return 0;
  return pc::tune_lookup(pc::tune_key(block_size, prec, n, nnz), shape) ? 1 : 0;
}

void pc_tune_clear(void) {
  {
    std::lock_guard<std::mutex> lk(pc::g_tmu);
    pc::g_cg.clear();
    pc::g_autoloaded = true;   // a cleared table stays empty until loaded again
  }
  pc_batch_clear_tuned();
}

pc_status pc_tune_save(const char* path) {
  if (!path || !path[0]) return PC_ERR_INVALID_ARG;
  std::string out;
  {
    std::lock_guard<std::mutex> lk(pc::g_tmu);
    char buf[512];
    for (const pc::CgEntry& e : pc::g_cg) {
      snprintf(buf, sizeof buf,
               "{\"kind\": \"cg\", \"bs\": %d, \"prec\": %d, \"log2n\": %d, \"log2deg\": %d, \"sms\": %d, "
               "\"spmv_ctas_per_sm\": %d, \"ring_stages\": %d, \"bin_pipe\": %d, \"fuse_update\": %d, "
               "\"us_per_iteration\": %.6g}\n",
               e.key.bs, e.key.prec, e.key.log2n, e.key.log2deg, e.key.sms, e.shape.spmv_ctas_per_sm,
               e.shape.ring_stages, e.shape.bin_pipe, e.shape.fuse_update, e.shape.us_per_iteration);
      out += buf;
    }
  }
  pc::batch_tune_lines(out);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return PC_ERR_INVALID_ARG;
  const bool ok = fwrite(out.data(), 1, out.size(), f) == out.size();
  if (fclose(f) != 0 || !ok) {
    remove(tmp.c_str());
    return PC_ERR_INVALID_ARG;
  }
  if (rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return PC_ERR_INVALID_ARG;
  }
  return PC_OK;
}

pc_status pc_tune_load(const char* path, int32_t* entries) {
  if (!path || !path[0]) return PC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(pc::g_tmu);
  int n = 0;
  const pc_status s = pc::load_locked(path, &n);
  if (entries) *entries = n;
  return s;
}

}  // extern "C"
