// Entry points of the stream engine used by the LSQR driver.
#pragma once

#include "qcpd_plan.h"


namespace qcpd {

// Builds the plan's stream layout on first use; *ok tells whether the engine
// can run the plan (zero, R+ and second-order-cone blocks of at most 256
// rows, magnitudes within the double-float range); when it cannot,
// qcp_last_error says why.
int stream_ready(qcp_plan* p, bool* ok);

// Runs the remaining LSQR iterations of systems [s0, s0 + ns) in one mode
// (0 JVP, 1 VJP), the range's active counter at `active`: converts the
// Krylov vectors to df64 pairs, iterates in chunks of check_every
// iterations (two launches per iteration, CUDA graphs), converts back.  Adds
// the device time of the chunks to p->pass_ms.
int iterate_stream(qcp_plan* p, int mode, int s0, int ns, int* active, bool scaled, const qcp_options& opts);

}  // namespace qcpd
