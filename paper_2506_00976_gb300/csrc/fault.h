// fault.h -- host-side fault injection for tests and the wait limit of the
// bounded device waits, both read from the environment.
//   QWB_FAULT="site=value[,site=value...]" with the sites
//     ns_pivot_cap=<k>          the network simplex stops after k pivots
//                               (QWB_ERR_NOT_CONVERGED unless already optimal)
//     ipf_bulk_skip_chunk=<c>   the bulk-copy IPF sweeps never issue chunk c,
//                               so its bounded wait runs out (QWB_ERR_TIMEOUT)
//   QWB_WAIT_TIMEOUT_MS=<ms>    limit of every bounded device wait (default 2000)
#pragma once
#include <cstdint>

namespace qwb {

// The value given for `site` in QWB_FAULT, or `def` when it is absent.
int64_t fault_param(const char* site, int64_t def);
// The bounded-wait limit in nanoseconds.
uint64_t wait_timeout_ns();

}  // namespace qwb
