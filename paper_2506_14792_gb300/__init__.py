"""GB300 (sm_103a) library for IMEX spectral timesteps and their exact discrete adjoints.

The compute path is the CUDA library ``libspadj.so`` (built in-tree by
``paper_2506_14792_gb300.build``); ``spadj`` is its ctypes binding.  There is no
CPU fallback: importing the binding without the library raises.
"""
