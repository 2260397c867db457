// Launch-shape autotuner of the LMA library.
//
// A tuning "site" is one kernel launch (or a short sequence) whose shape has
// several valid choices — the number of window groups of the summary Gram,
// the variant of the support-set projection, the width of the sweep's
// intermediate panel update.  For a site and a shape class (its key: the
// site's name plus the sizes that decide the best choice), pick() times each
// candidate on the caller's own data with CUDA events on the caller's stream
// and keeps the fastest; the choice is cached per device for the life of the
// process and, when LMA_TUNE_CACHE names a file, in that file (one line per
// entry: device name, key, choice), which later processes read back.
//
// Only launches that can be repeated without changing the result are tuned
// on live data (they read their inputs and overwrite their outputs).  With
// LMA_AUTOTUNE=0 (or lma_autotune(0)) every site takes the shape its model
// predicts (the `fallback` argument).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

namespace lma {
namespace tune {

// Whether sites are timed (default: on; LMA_AUTOTUNE=0 or set_enabled(false) turns it off).
bool enabled();
void set_enabled(bool on);

// The cached choice for key, or, if none: time run(c) for every candidate c
// (one warm-up launch and `reps` timed launches each, on stream st), cache and
// return the fastest.  Without tuning: `fallback`.  run() must be repeatable.
int pick(const std::string& key, const std::vector<int>& cands, int fallback, cudaStream_t st,
         const std::function<void(int)>& run, int reps = 2);

// Pins every key starting with `prefix` to `choice` (where it is a
// candidate), ahead of the cache and of timing; the latest matching pin wins.
// prefix == nullptr removes all pins.
void pin(const char* prefix, int choice);

// Text report of the cache: "device | key | choice | candidates and their ms".
std::string report();
void clear();

}  // namespace tune
}  // namespace lma
