// Tuning cache of MOLC_AUTOTUNE: the launch configuration chosen for a plan, kept in a JSON file so that a later
// plan with the same signature, on the same kind of device and with the same library build, takes it without
// timing anything.  Host code only.
#pragma once

#include <string>
#include <vector>

namespace molc {

struct TuneRecord {
  std::string key;      // plan signature: what molc_create was given that decides the plan's kernels
  std::string device;   // device name, SM count and compute capability
  std::string build;    // library build identifier (hash of the sources it was compiled from)
  int sweep_depth = 0;  // bundle FP32 sweep: staging depth (0: not a bundle plan)
  int tile_cells = 0, tile_groups = 0, block_threads = 0;   // tiled FP32 sweep (0: not a tiled plan)
  double best_ms = 0;   // time of one sweep launch in the chosen configuration when it was tuned
};

// The records of a cache file's text; false, with the reason, when the text is not a cache this library wrote.
bool tune_parse(const std::string &text, std::vector<TuneRecord> &out, std::string &why);
// The JSON text of a cache holding `recs`.
std::string tune_serialize(const std::vector<TuneRecord> &recs);

// Process-wide cache file.  tune_cache_set: read `path` (a missing file is an empty cache); nullptr or "" switches
// the cache off.  Returns the records read, or -1 (setting unchanged) with the reason.
int tune_cache_set(const char *path, std::string &why);
bool tune_cache_enabled();
// The record for (key, device, build), if the cache holds one.
bool tune_cache_lookup(const std::string &key, const std::string &device, const std::string &build, TuneRecord &out);
// Add or replace the record of rec's (key, device, build) and rewrite the file (merged with what another process
// may have added since it was read; written to a temporary file, then renamed over the cache).
bool tune_cache_store(const TuneRecord &rec, std::string &why);

}  // namespace molc
