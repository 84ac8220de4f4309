// Tuned schedules of the two-site update, written by paper_2609_18841_b300/autotune.py
// from timings on the device (NVIDIA B300 SXM6 AC); no entry: the defaults of lindtebd.h.
#pragma once

struct LtSchedule {
  int d, precision, chi_max;          // values per site, lt_precision, chi_max
  int theta_path, env_ctas_per_sm;
};

static const LtSchedule kLtSchedules[] = {
    {2, 1, 16, 2, 8},  // 12.0 -> 11.8 ms per step
    {2, 1, 32, 1, 8},  // 25.6 -> 25.6 ms per step
    {2, 1, 64, 1, 8},  // 73.1 -> 73.1 ms per step
    {2, 1, 128, 1, 8},  // 386.8 -> 386.8 ms per step
    {2, 1, 256, 1, 8},  // 2594.4 -> 2594.4 ms per step
    {2, 0, 16, 1, 8},  // 100.9 -> 100.9 ms per step
    {2, 0, 32, 1, 8},  // 288.4 -> 288.4 ms per step
    {2, 0, 64, 1, 8},  // 1517.0 -> 1517.0 ms per step
    {2, 0, 128, 1, 8},  // 1954.6 -> 1954.6 ms per step
    {2, 0, 256, 1, 8},  // 13023.3 -> 13023.3 ms per step
    {4, 1, 16, 1, 8},  // 3.9 -> 3.9 ms per step
    {4, 1, 32, 1, 8},  // 10.3 -> 10.3 ms per step
    {4, 1, 64, 1, 8},  // 101.9 -> 101.9 ms per step
    {4, 1, 128, 1, 8},  // 407.7 -> 407.7 ms per step
    {4, 0, 16, 1, 8},  // 52.0 -> 52.0 ms per step
    {4, 0, 32, 1, 8},  // 276.3 -> 276.3 ms per step
    {4, 0, 64, 1, 8},  // 2160.9 -> 2160.9 ms per step
    {4, 0, 128, 1, 8},  // 10950.6 -> 10950.6 ms per step
};
