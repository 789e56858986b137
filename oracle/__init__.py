"""CPU oracle (test infrastructure only): a plain FP64 restatement of RQI-PCGTLS.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
use this package. It shares no code with the CUDA library. Import the submodule
``oracle.rqi_pcgtls``.
"""
