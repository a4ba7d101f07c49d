"""GB300-native FNR impulse filter for infrared frames (arXiv 1201.3972).

The compute path is the C-ABI library built from ``csrc/`` (libirfnr.so);
``_lib`` is its thin ctypes binding. Importing the package does not load the
library; the first call that needs it does, and raises if it is missing.
"""
from ._lib import (IR_ALGO_AUTO, IR_ALGO_BITPLANE, IR_ALGO_DENSE, IR_ALGO_DENSE3, IR_ALGO_NETWORK, IR_U8, IR_U14,
                   IR_U16, BatchPlan, Filter, IrError, load)

__all__ = ["Filter", "BatchPlan", "IrError", "load", "IR_U8", "IR_U16", "IR_U14", "IR_ALGO_AUTO",
           "IR_ALGO_DENSE3", "IR_ALGO_NETWORK", "IR_ALGO_BITPLANE", "IR_ALGO_DENSE", "synth"]
