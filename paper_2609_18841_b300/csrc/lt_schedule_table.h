// Tuned schedules of the two-site update, written by paper_2609_18841_b300/autotune.py
// from timings on the device (no entry: the defaults of lindtebd.h).
#pragma once

struct LtSchedule {
  int d, precision, chi_max;          // values per site, lt_precision, chi_max
  int theta_path, jacobi_epp, env_ctas_per_sm;
};

static const LtSchedule kLtSchedules[] = {
    {0, -1, 0, 0, 0, 0},  // placeholder: matches no context
};
