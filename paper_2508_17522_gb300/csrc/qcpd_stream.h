// Entry points of the stream engine used by the LSQR driver.
#pragma once

#include "qcpd_plan.h"


namespace qcpd {

// Builds the plan's stream layout on first use; *ok tells whether the engine
// can run the plan (zero, R+ and second-order-cone blocks of at most 256
// rows, magnitudes within the double-float range); when it cannot,
// qcp_last_error says why.
int stream_ready(qcp_plan* p, bool* ok);

// Builds once the dense D Pi of the plan's exponential, power and PSD blocks
// as df64 matrices (p->d_dpi, row-major, at p->d_dpi_off[block] for each
// coupled block, -1 for SOC blocks): exponential and power blocks copy
// their stored 3 x 3, a PSD block applies the pass engine's map to each unit
// vector of its entries.  *ok false (p->dpi_why says why) for a PSD block of
// more than 256 entries, more than 2 GB of matrices, or an entry above the
// double-float range.  The stream and cluster engines apply them.
int dense_dpi_ready(qcp_plan* p, bool* ok);

// Runs the remaining LSQR iterations of systems [s0, s0 + ns) in one mode
// (0 JVP, 1 VJP), the range's active counter at `active`: converts the
// Krylov vectors to df64 pairs, iterates in chunks of check_every
// iterations (two launches per iteration, CUDA graphs), converts back.  Adds
// the device time of the chunks to p->pass_ms.
int iterate_stream(qcp_plan* p, int mode, int s0, int ns, int* active, bool scaled, const qcp_options& opts);

// Whether the JVP range [sa0, sa0 + ns) and the VJP range [sb0, sb0 + ns)
// can iterate in step: system sa0 + i and system sb0 + i on one problem (a
// plan that is not a batch plan).
bool stream_can_pair(const qcp_plan* p, int sa0, int sb0, int ns);

// Runs the remaining LSQR iterations of the JVP range and the VJP range in
// step: the VJP systems' first u-pass alone, then launches that each run one
// product (with G, then with G^T) for both systems of every pair, reading
// M's slots once for the two; each range's active counter at active_a /
// active_b.  Adds the device time to p->pass_ms and the system passes that
// shared a read of M to p->shared_passes.
int iterate_stream_pair(qcp_plan* p, int sa0, int sb0, int ns, int* active_a, int* active_b, bool scaled,
                        const qcp_options& opts);

}  // namespace qcpd
