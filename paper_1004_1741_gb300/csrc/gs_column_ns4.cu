// Column-march Gauss-Seidel with 4 sweeps per task (gs_column_ns.cuh), instantiated in a translation unit of
// its own so that the NS variants compile in parallel.
#include "gs_column_ns.cuh"

STN_COLUMN_NS_INSTANTIATE(4)
