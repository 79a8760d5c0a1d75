"""GB300-native EPIC (E-field Parallel Imaging Correlator) imaging hot path.

The compute path is the C-ABI CUDA library ``libepic.so`` (built for sm_103a);
``paper_2301_09662_gb300.epic`` is its thin Python binding and ``synth`` makes
seeded synthetic inputs.
"""
