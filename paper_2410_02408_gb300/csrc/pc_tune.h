// Launch-shape table of the CG graph engine and its cache file (pc_tune.cu); internal.
#pragma once
#include <stdint.h>

#include <map>
#include <string>

#include "pc.h"

namespace pc {

struct TuneKey {
  int32_t bs, prec, log2n, log2deg, sms;
};

// SM count of the current device (0 when no device answers).
int32_t current_sms();
// Key of a system: block size, precision, ceil(log2 n), round(log2(nnz / n)), SM count.
TuneKey tune_key(int32_t bs, int32_t prec, int64_t n, int64_t nnz);
// Loads the file named by PC_TUNE_CACHE once per process (no effect when unset).
void tune_autoload();
bool tune_lookup(const TuneKey& k, pc_shape* out);
void tune_record(const TuneKey& k, const pc_shape& s);
// Saves the table to PC_TUNE_CACHE when it is set.
pc_status tune_save_env();

// pc_batched.cu: the batched launch shapes in the same file.
bool batch_tune_parse(const std::map<std::string, std::string>& kv);
void batch_tune_lines(std::string& out);

}  // namespace pc
