// Tuned schedules of the two-site update, written by paper_2609_18841_b300/autotune.py
// from timings on the device (NVIDIA B300 SXM6 AC); no entry: the defaults of lindtebd.h.
#pragma once

struct LtSchedule {
  int d, precision, chi_max;          // values per site, lt_precision, chi_max
  int theta_path, env_ctas_per_sm;
};

static const LtSchedule kLtSchedules[] = {
    {2, 1, 16, 2, 4},  // 14.6 -> 13.4 ms per step
    {2, 1, 32, 1, 8},  // 28.5 -> 28.5 ms per step
    {2, 1, 64, 1, 8},  // 82.1 -> 82.1 ms per step
    {2, 1, 128, 1, 8},  // 600.7 -> 600.7 ms per step
    {2, 1, 256, 1, 8},  // 4596.8 -> 4596.8 ms per step
    {2, 0, 16, 1, 8},  // 100.4 -> 100.4 ms per step
    {2, 0, 32, 1, 8},  // 288.2 -> 288.2 ms per step
    {2, 0, 64, 1, 8},  // 1518.2 -> 1518.2 ms per step
    {2, 0, 128, 1, 8},  // 1892.7 -> 1892.7 ms per step
    {2, 0, 256, 1, 8},  // 12678.4 -> 12678.4 ms per step
    {4, 1, 16, 1, 8},  // 4.1 -> 4.1 ms per step
    {4, 1, 32, 1, 8},  // 11.5 -> 11.5 ms per step
    {4, 1, 64, 1, 8},  // 240.6 -> 240.6 ms per step
    {4, 1, 128, 1, 8},  // 1098.5 -> 1098.5 ms per step
    {4, 0, 16, 1, 8},  // 52.0 -> 52.0 ms per step
    {4, 0, 32, 1, 8},  // 276.7 -> 276.7 ms per step
    {4, 0, 64, 1, 8},  // 2095.7 -> 2095.7 ms per step
    {4, 0, 128, 1, 8},  // 10585.4 -> 10585.4 ms per step
};
