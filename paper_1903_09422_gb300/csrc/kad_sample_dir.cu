// The block-per-sample kernel built for directed graphs (Section 5: KADABRA
// also covers directed graphs): the s side expands along out-arcs and traces
// back over in-arcs, the t side the other way round.  kad_launch_sample hands a
// directed graph's launches to kad_launch_sample_directed defined here.
#define KAD_DIRECTED 1
#include "kad_sample.cu"
