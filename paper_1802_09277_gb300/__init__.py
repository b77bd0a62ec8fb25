"""GB300-native space-time multigrid for the dG-IgA heat equation
(Hofer, Langer, Neumueller, arXiv:1802.09277).

The compute path is the CUDA/C++ library ``libst_iga.so`` behind the C ABI in
``include/st_iga.h``; ``paper_1802_09277_gb300.st`` is its thin ctypes
binding.  Importing the package does not load the library; ``st.load()``
does, and fails loudly when it is missing.
"""
