// The warp-per-sample kernel built for directed graphs (Section 5: KADABRA also
// covers directed graphs); kad_launch_wsample hands a directed graph's launches
// to kad_launch_wsample_directed defined here.
#define KAD_DIRECTED 1
#include "kad_wsample.cu"
