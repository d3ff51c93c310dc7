// Entry points of the cluster engine used by the LSQR driver.
#pragma once

#include "qcpd_cluster.cuh"
#include "qcpd_cluster_df.cuh"
#include "qcpd_plan.h"

namespace qcpd {

// Builds (once per requested cluster size) the cluster layouts of the plan's
// problems; *ok tells whether every problem fits the shared-memory limit.
int cluster_ready(qcp_plan* p, int nsys, bool* ok);

// Runs the remaining LSQR iterations of systems [0, nsys) with one cluster
// per system, one launch per cluster size present; adds the device time to
// p->pass_ms.
template <typename T>
int iterate_cluster(qcp_plan* p, int mode, int nsys, const PlanView<T>& v, const qcp_options& opts);

}  // namespace qcpd
