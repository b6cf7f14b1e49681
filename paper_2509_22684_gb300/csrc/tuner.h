// tuner.h -- schedule cache of the autotuner.
//
// The paper calls for tools that adapt the kernels' runtime parameters to the
// GPU they run on (Section V-A).  An entry records, for one (GPU, field,
// log_n, direction), the digit split into passes, the columns per block of
// each pass and the twiddle mode that timed fastest.  Entries live in memory
// and, when ZKNTT_TUNE_CACHE names a file, in that file as one JSON object per
// line.
#pragma once

namespace zkntt {

struct TuneEntry {
    int passes = 0;
    int digits[4] = {0, 0, 0, 0};
    int log_cols[4] = {-1, -1, -1, -1};
    int mode = 0;
    int ilp = 0;
    double ms = 0.0;
};

bool tuner_lookup(int field, int log_n, int dir, TuneEntry *out);
void tuner_store(int field, int log_n, int dir, const TuneEntry &e);

}  // namespace zkntt
