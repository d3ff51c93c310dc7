// Entry points of the cluster engine used by the LSQR driver.
#pragma once

#include "qcpd_cluster.cuh"
#include "qcpd_cluster_df.cuh"
#include "qcpd_plan.h"

namespace qcpd {

// Builds (once per requested cluster size) the cluster layouts of the plan's
// problems; *ok tells whether every problem fits the shared-memory limit
// (and, with need_df, whether the double-float kernel can run the plan:
// LSMR has no FP64 cluster kernel).
int cluster_ready(qcp_plan* p, int nsys, bool* ok, bool need_df = false);

// A range of systems [s0, s0 + ns) iterating one mode (0 JVP, 1 VJP);
// seg is its index in the call (its active counter).
struct ClusterSeg {
    int mode, s0, ns, seg;
};

// Runs the remaining LSQR iterations of the given system ranges with one
// cluster per system, one launch per (range, cluster size).  The first
// range's launches go to the plan's stream, the others to a second stream
// forked from it and joined back, so a JVP range and a VJP range run side by
// side.  nsys_call (all systems of the call) sets the automatic cluster size.
// Adds the device time to p->pass_ms.
template <typename T>
int iterate_cluster(qcp_plan* p, const ClusterSeg* segs, int nseg, int nsys_call, const PlanView<T>& v,
                    const qcp_options& opts);

}  // namespace qcpd
