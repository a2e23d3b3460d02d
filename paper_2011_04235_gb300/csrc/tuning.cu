// Tuning table: the parameters the autotuner (paper_2011_04235_gb300/autotune.py)
// picks on the GPU and the library reads.
//
// A plain-text file, one entry per line ('#' starts a comment):
//   core  <n_max> <panel> <parts> <resident> <fast>
//         FP32 core SVD of an n x n core, n <= n_max (first matching line):
//         panel 16 | 32, parts 0..8 CTAs per cluster, resident 0 | 1,
//         fast 0 | 1 (the Gram sweep with one barrier per inner round and
//         fast rotations)
//   chunk <prec> <phase> <k_max> <c>
//         border rows (phase 0, Eq. 2) / columns (phase 1, Eq. 3) appended per
//         incremental step when the caller passes 0, for a phase whose target
//         rank is <= k_max; prec 0 = FP64, 1 = mixed
//   bucket <prec> <dim_max> <class>
//         batched Jacobi of the A11 blocks: problems whose longer side is
//         <= dim_max run in the register-tile class `class` (never below the
//         class their size needs)
//   gemm <tc_min_flops>
//         the mixed form's FP32 products of at least this many flops
//         (2 M N K) run on the tensor cores, smaller ones on the SIMT kernel
// The file is read on first use from $FASTPI_TUNING, else from tuning.txt next
// to libfastpi.so; without one the built-in defaults apply (chunk 256, core
// tiling by the SM count, natural bucket classes).
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "jacobi.cuh"
#include "tuning.cuh"

namespace fastpi {
namespace {

struct CoreRow {
  int n_max, panel, parts, resident, fast;
};
struct ChunkRow {
  int prec, phase;
  int64_t k_max, c;
};
struct BucketRow {
  int prec, dim_max, cls;
};

struct Table {
  bool loaded = false;
  std::string source = "built-in defaults";
  std::vector<CoreRow> core;
  std::vector<ChunkRow> chunk;
  std::vector<BucketRow> bucket;
  double tc_min_flops = 0;   // 0: not in the table
};

std::mutex g_mu;
Table g_tab;

std::string default_path() {
  const char* e = std::getenv("FASTPI_TUNING");
  if (e && *e) return e;
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&default_path), &info) && info.dli_fname) {
    std::string so = info.dli_fname;
    const size_t slash = so.rfind('/');
    return (slash == std::string::npos ? std::string(".") : so.substr(0, slash)) + "/tuning.txt";
  }
  return "tuning.txt";
}

// Parses `path` into t; false (t untouched) when the file cannot be read or a
// line is malformed.
bool parse(const std::string& path, Table& t, std::string* why) {
  std::ifstream in(path);
  if (!in) {
    if (why) *why = "cannot open " + path;
    return false;
  }
  Table out;
  std::string line;
  int ln = 0;
  while (std::getline(in, line)) {
    ++ln;
    const size_t hash = line.find('#');
    if (hash != std::string::npos) line.resize(hash);
    std::istringstream ss(line);
    std::string kind;
    if (!(ss >> kind)) continue;
    bool ok = false;
    if (kind == "core") {
      CoreRow r;
      ok = bool(ss >> r.n_max >> r.panel >> r.parts >> r.resident >> r.fast) && (r.panel == 16 || r.panel == 32) &&
           r.parts >= 0 && r.parts <= 8 && r.n_max >= 2;
      if (ok) out.core.push_back(r);
    } else if (kind == "chunk") {
      ChunkRow r;
      ok = bool(ss >> r.prec >> r.phase >> r.k_max >> r.c) && (r.prec == 0 || r.prec == 1) &&
           (r.phase == 0 || r.phase == 1) && r.c >= 1;
      if (ok) out.chunk.push_back(r);
    } else if (kind == "gemm") {
      double v = 0;
      ok = bool(ss >> v) && v >= 1.0;
      if (ok) out.tc_min_flops = v;
    } else if (kind == "bucket") {
      BucketRow r;
      ok = bool(ss >> r.prec >> r.dim_max >> r.cls) && (r.prec == 0 || r.prec == 1) && r.cls >= 0 && r.cls <= 4;
      if (ok) out.bucket.push_back(r);
    }
    if (!ok) {
      if (why) *why = path + ":" + std::to_string(ln) + ": malformed line";
      return false;
    }
  }
  out.loaded = true;
  out.source = path;
  t = std::move(out);
  return true;
}

const Table& table() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_tab.loaded) {
    Table t;
    if (!parse(default_path(), t, nullptr)) {
      t = Table{};
      t.loaded = true;
    }
    g_tab = std::move(t);
  }
  return g_tab;
}

}  // namespace

bool tuned_core_tiling(int n, CoreTiling* out) {
  const Table& t = table();
  for (const CoreRow& r : t.core)
    if (n <= r.n_max) {
      out->panel = r.panel;
      out->parts = r.parts;
      out->resident = r.resident != 0;
      out->fast_solve = r.fast != 0;
      return true;
    }
  return false;
}

int64_t tuned_chunk(int prec, int phase, int64_t k_target, int64_t fallback) {
  const Table& t = table();
  for (const ChunkRow& r : t.chunk)
    if (r.prec == prec && r.phase == phase && k_target <= r.k_max) return r.c;
  return fallback;
}

int tuned_bucket_class(int prec, int dim, int natural) {
  const Table& t = table();
  for (const BucketRow& r : t.bucket)
    if (r.prec == prec && dim <= r.dim_max) return r.cls > natural ? r.cls : natural;
  return natural;
}

bool load_tuning(const char* path, std::string* why) {
  Table t;
  if (!path) {
    t.loaded = true;
  } else if (!parse(path, t, why)) {
    return false;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_tab = std::move(t);
  return true;
}

double tuned_tc_min_flops(double fallback) {
  const Table& t = table();
  return t.tc_min_flops > 0 ? t.tc_min_flops : fallback;
}

std::string tuning_source() { return table().source; }

}  // namespace fastpi
